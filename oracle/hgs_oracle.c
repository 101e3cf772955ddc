/*
 * hgs_oracle.c -- plain FP64 CPU oracle for the hybrid 2D/3D Gaussian
 * rasterizer of EGGS (Exchangeable 2D/3D Gaussian Splatting).
 *
 * TEST INFRASTRUCTURE ONLY.  The product path never calls, links or loads this
 * file.  Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of
 * bench.py use it.  It shares no code, header, table or helper with the CUDA
 * path under paper_2512_02932_gb300/csrc.
 *
 * What it computes (each function cites the passage it follows):
 *   (1) orc_prepare / orc_render -- per pixel, in double precision, over every
 *       primitive: the unified distance d of Eq. 1 (Sec. 3.1), the
 *       contribution alpha*exp(-d/2) (Sec. 3.1), and front-to-back
 *       alpha-blending (Eq. 2).  3D Gaussians use the affine (EWA) projection
 *       of App. C, Eq. 13; 2D Gaussians use the ray-splat intersection of
 *       App. C, Eqs. 14-15, which this oracle obtains by solving the 3x3
 *       ray/plane system directly (Gaussian elimination), not by Eq. 14's
 *       closed form.  The only acceleration is a uniform grid over
 *       conservative bounding boxes, which cannot change the result.
 *   (2) orc_contract_bin -- an FP32 replica of the binning contract: the
 *       written sequence of single-precision operations that decides each
 *       primitive's tile rectangle and 32-bit depth key.  Tile lists built
 *       from it are compared bit for bit with the GPU's.
 *   (3) orc_sh_basis -- the real spherical-harmonic basis (degree <= 3) that
 *       decodes view-dependent colour from f (Sec. 3.1).
 *   (4) orc_exchange -- Adaptive Type Exchange: effective rank (Eq. 3), the
 *       3D->2D permutation reparameterisation (Eqs. 4-5, App. D Eqs. 17-19)
 *       and the 2D->3D flag flip (Sec. 3.2).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (see build.py).
 * -ffp-contract=off is required: the FP32 contract must round every
 * multiply and add separately.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* configuration indices (double array passed from Python)                  */
/* ------------------------------------------------------------------------ */
enum {
  CF_NEAR = 0, CF_ALPHA_MIN, CF_ALPHA_MAX, CF_T_MIN, CF_LAMBDA_Z, CF_THETA_Z,
  CF_T_Z, CF_DILATION, CF_BG0, CF_BG1, CF_BG2, CF_COUNT
};

/* Threshold decisions.  Eq. 2 with the contribution rule of Sec. 3.1 takes
 * three kinds of discrete decision per (pixel, primitive) pair: does the pair
 * clear alpha_min, does a surfel's hit lie beyond the near plane, and does
 * the pixel stop before it (T' < T_min); the normal map adds the sign that
 * turns a primitive's normal to the camera.  Where the FP64 value sits within
 * a band around the threshold that a binary32 evaluation could cross, the
 * decision is ambiguous: both outcomes are correct results of the method
 * evaluated in binary32.  The renderer then enumerates the outcomes of the
 * ambiguous decisions met before the pixel terminates, depth first, up to
 * ORC_MAXV results ("variants"); a pixel with more is reported as not
 * comparable.  (A stop decision ends the walk, so a run of ambiguous stops
 * over consecutive faint contributors adds one result each, not a doubling.)  In binary32 a contribution alpha*exp(-d/2) carries a
 * relative error of about 1e-5 (d ~ 11 near the cutoff), and the
 * transmittance after a few hundred contributors about 1e-4; the bands are
 * five to ten times wider. */
#define AMB_ALPHA_REL 5e-5   /* |alpha*G - alpha_min| <= this * alpha_min  */
#define AMB_T_REL     1e-3   /* |T' - T_min| <= this * T_min               */
#define AMB_NEAR_REL  1e-5   /* |z - near| <= this * max(1, near)          */
#define AMB_FLIP      1e-5   /* |n . mu_c| / |mu_c| below this             */
#define ORC_MAXDEC    31   /* decisions along one path (bits of the choice word) */
#define ORC_MAXV      64   /* results enumerated per pixel */
/* An ambiguous alpha_min decision whose whole weight alpha T is at most
 * ORC_FAINT moves the pixel's outputs by at most that weight times the
 * magnitudes involved (a few 1e-6, far below the 1e-3 image tolerance): it is
 * taken the FP64 way and its effect added to the tolerance (and one to the
 * contributor count's slack) instead of doubling the results. */
#define ORC_FAINT     2e-6
/* Conditioning.  In binary32, (u, v) evaluated from the pixel's offset to
 * the projected centre carry an error of up to COND_ULPS ulps of the
 * magnitude of the terms that cancel, |du/dx dx| + |du/dy dy| (likewise v):
 * a few ulps for the record's coefficients and two for the evaluation.  That
 * bounds the error of each contribution (dag below); the renderer carries it
 * through Eq. 2 as a per-channel tolerance on the pixel's result, and widens
 * the alpha_min and T_min bands by it.  It is negligible except for extremely
 * anisotropic footprints evaluated far from their centre (e.g. a 1e5:1
 * ribbon thousands of pixels along its length). */
#define COND_ULPS     8.0
#define EPS32         5.960464477539063e-08

/* ------------------------------------------------------------------------ */
/* (3) real spherical harmonics, degree <= 3                                 */
/* Real basis built from the complex Y_l^m (with Condon-Shortley phase):     */
/*   m>0: sqrt2 Re Y_l^m, m<0: sqrt2 Im Y_l^|m|, m=0: Y_l^0, index l*l+l+m.  */
/* ------------------------------------------------------------------------ */
static void sh_basis(int deg, double x, double y, double z, double *Y) {
  const double PI = 3.14159265358979323846;
  Y[0] = 0.5 * sqrt(1.0 / PI);
  if (deg < 1) return;
  const double k1 = sqrt(3.0 / (4.0 * PI));
  Y[1] = -k1 * y;
  Y[2] = k1 * z;
  Y[3] = -k1 * x;
  if (deg < 2) return;
  const double k2a = 0.5 * sqrt(15.0 / PI);
  const double k2b = 0.25 * sqrt(5.0 / PI);
  const double k2c = 0.25 * sqrt(15.0 / PI);
  Y[4] = k2a * x * y;
  Y[5] = -k2a * y * z;
  Y[6] = k2b * (2.0 * z * z - x * x - y * y);
  Y[7] = -k2a * x * z;
  Y[8] = k2c * (x * x - y * y);
  if (deg < 3) return;
  const double k3a = 0.25 * sqrt(35.0 / (2.0 * PI));
  const double k3b = 0.5 * sqrt(105.0 / PI);
  const double k3c = 0.25 * sqrt(21.0 / (2.0 * PI));
  const double k3d = 0.25 * sqrt(7.0 / PI);
  const double k3e = 0.25 * sqrt(105.0 / PI);
  Y[9] = -k3a * y * (3.0 * x * x - y * y);
  Y[10] = k3b * x * y * z;
  Y[11] = -k3c * y * (4.0 * z * z - x * x - y * y);
  Y[12] = k3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
  Y[13] = -k3c * x * (4.0 * z * z - x * x - y * y);
  Y[14] = k3e * z * (x * x - y * y);
  Y[15] = -k3a * x * (x * x - 3.0 * y * y);
}

void orc_sh_basis(int deg, int64_t n, const double *dirs, double *out) {
  const int nb = (deg + 1) * (deg + 1);
  for (int64_t i = 0; i < n; ++i) {
    double Y[16];
    sh_basis(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Y);
    for (int k = 0; k < nb; ++k) out[i * nb + k] = Y[k];
  }
}

/* ------------------------------------------------------------------------ */
/* quaternion (w, x, y, z), Hamilton convention, to rotation matrix          */
/* ------------------------------------------------------------------------ */
static void quat_to_rot(const double q[4], double R[9]) {
  double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------ */
/* (2) FP32 binning contract replica.  Every operation is a separately      */
/* rounded binary32 operation (this file is compiled with                   */
/* -ffp-contract=off); the order of operations is the contract.             */
/* ------------------------------------------------------------------------ */
static float f32_from_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t bits_from_f32(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* contract exp: Cody-Waite reduction x = k ln2 + r, |r| <= ln2/2, then the
 * degree-7 Taylor polynomial of e^r by Horner's rule, scaled by 2^k. */
float orc_c_exp(float x) {
  if (x != x) return x;
  if (x < -87.0f) return 0.0f;
  if (x > 88.0f) x = 88.0f;
  const float LOG2E = 0x1.715476p+0f;
  const float LN2_HI = 0x1.62e4p-1f;   /* 16 significant bits: k*LN2_HI exact */
  const float LN2_LO = 0x1.7f7d1cp-20f; /* ln2 - LN2_HI rounded to binary32 */
  float k = rintf(x * LOG2E);
  float r = x - k * LN2_HI;
  r = r - k * LN2_LO;
  /* Taylor coefficients 1/n!, n = 7..0, rounded to binary32 */
  float p = 0x1.a01a02p-13f;
  p = p * r + 0x1.6c16c2p-10f;
  p = p * r + 0x1.111112p-7f;
  p = p * r + 0x1.555556p-5f;
  p = p * r + 0x1.555556p-3f;
  p = p * r + 0.5f;
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  int ki = (int)k;
  float scale = f32_from_bits((uint32_t)(ki + 127) << 23);
  return p * scale;
}

/* contract log for normal x > 0: x = m 2^e with m in (sqrt(1/2), sqrt(2)],
 * ln m = 2 atanh(t), t = (m-1)/(m+1), atanh by its odd series to t^13. */
float orc_c_log(float x) {
  if (!(x > 0.0f)) return -INFINITY;
  uint32_t b = bits_from_f32(x);
  int e = (int)((b >> 23) & 0xff) - 127;
  float m = f32_from_bits((b & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) { m = m * 0.5f; e = e + 1; }
  float t = (m - 1.0f) / (m + 1.0f);
  float t2 = t * t;
  /* atanh(t)/t = sum t^(2k)/(2k+1), coefficients rounded to binary32 */
  float s = 0x1.3b13b2p-4f;
  s = s * t2 + 0x1.745d18p-4f;
  s = s * t2 + 0x1.c71c72p-4f;
  s = s * t2 + 0x1.24924ap-3f;
  s = s * t2 + 0x1.99999ap-3f;
  s = s * t2 + 0x1.555556p-2f;
  s = s * t2 + 1.0f;
  float lnm = (2.0f * t) * s;
  float fe = (float)e;
  return fe * 0x1.62e4p-1f + (fe * 0x1.7f7d1cp-20f + lnm);
}

static float pad_f(float r) { return r * 1.0009765625f + 0.015625f; }

#define ORC_ROWP 12 /* tile-set parameters per primitive */

/* pixel-centre coverage of [lo, hi] -> inclusive pixel range, then tiles */
static int c_range(float lo, float hi, int extent, int tile, int *t0, int *t1) {
  float flo = lo - 0.5f, fhi = hi - 0.5f;
  if (!(flo <= fhi)) return 0;
  flo = fmaxf(flo, -1.0f);
  fhi = fminf(fhi, (float)extent);
  int p0 = (int)ceilf(flo), p1 = (int)floorf(fhi);
  if (p0 < 0) p0 = 0;
  if (p1 > extent - 1) p1 = extent - 1;
  if (p0 > p1) return 0;
  *t0 = p0 / tile;
  *t1 = p1 / tile;
  return 1;
}

/* One primitive through the contract.  cam: R[9] t[3] fx fy cx cy.
 * Returns 1 and fills rect {tx0,tx1,ty0,ty1}, depth bits and the tile-set
 * parameters rowp (ORC_ROWP floats, row_span) if binned. */
static int contract_one(const float mu[3], const float ls[3], const float q[4],
                        float logit, int type, const float *cam, int W, int H,
                        int tile, float near_z, float alpha_min, float dil,
                        int rect[4], uint32_t *dbits, float rowp[ORC_ROWP]) {
  const float *Rc = cam, *tc = cam + 9;
  const float fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
  float X = ((Rc[0] * mu[0] + Rc[1] * mu[1]) + Rc[2] * mu[2]) + tc[0];
  float Y = ((Rc[3] * mu[0] + Rc[4] * mu[1]) + Rc[5] * mu[2]) + tc[1];
  float Z = ((Rc[6] * mu[0] + Rc[7] * mu[1]) + Rc[8] * mu[2]) + tc[2];
  *dbits = bits_from_f32(Z);
  if (!(Z > near_z)) return 0;
  float alpha = 1.0f / (1.0f + orc_c_exp(-logit));
  if (!(alpha >= alpha_min)) return 0;
  float dmax = 2.0f * orc_c_log(alpha / alpha_min);
  float sx = orc_c_exp(ls[0]), sy = orc_c_exp(ls[1]), sz = orc_c_exp(ls[2]);
  float qq = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
  if (!(qq > 0.0f)) return 0;
  float inv = 1.0f / sqrtf(qq);
  float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
  float Rq[9];
  Rq[0] = 1.0f - 2.0f * (y * y + z * z);
  Rq[1] = 2.0f * (x * y - w * z);
  Rq[2] = 2.0f * (x * z + w * y);
  Rq[3] = 2.0f * (x * y + w * z);
  Rq[4] = 1.0f - 2.0f * (x * x + z * z);
  Rq[5] = 2.0f * (y * z - w * x);
  Rq[6] = 2.0f * (x * z - w * y);
  Rq[7] = 2.0f * (y * z + w * x);
  Rq[8] = 1.0f - 2.0f * (x * x + y * y);
  float a[3][3]; /* a[k][i]: camera-space axis k, component i */
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      a[k][i] = (Rc[3 * i + 0] * Rq[0 * 3 + k] + Rc[3 * i + 1] * Rq[1 * 3 + k]) +
                Rc[3 * i + 2] * Rq[2 * 3 + k];
  float iz = 1.0f / Z;
  float xz = X * iz, yz = Y * iz;
  float ctrx, ctry, hx, hy;
  /* tile set: the footprint is the ellipse with centre (ctrx, ctry) and
   * half extents hx, hy; its horizontal chord at height y is centred on
   * ctrx + kslope (y - ctry) with half length wch sqrt(1 - ((y - ctry)/hy)^2),
   * and its leftmost (rightmost) point lies at y = ctry - yoff (+ yoff) */
  float kslope = 0.0f, wch = 0.0f, yoff = 0.0f;
  int full = 0;
  int whole = 0;
  /* a surfel whose disc reaches the near plane (or whose image conic is
   * degenerate): the disc in pixel-homogeneous camera coordinates */
  int disc = 0;
  float dP[3] = {0.0f, 0.0f, 0.0f}, dA[3] = {0.0f, 0.0f, 0.0f}, dB[3] = {0.0f, 0.0f, 0.0f};
  if (type == 1) {
    float c0 = sx * sx, c1 = sy * sy, c2 = sz * sz;
    float V[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        V[i][j] = (c0 * (a[0][i] * a[0][j]) + c1 * (a[1][i] * a[1][j])) +
                  c2 * (a[2][i] * a[2][j]);
    float j00 = fx * iz, j02 = -(j00 * xz);
    float j11 = fy * iz, j12 = -(j11 * yz);
    float t00 = j00 * V[0][0] + j02 * V[2][0];
    float t01 = j00 * V[0][1] + j02 * V[2][1];
    float t02 = j00 * V[0][2] + j02 * V[2][2];
    float t11 = j11 * V[1][1] + j12 * V[2][1];
    float t12 = j11 * V[1][2] + j12 * V[2][2];
    float s00 = (j00 * t00 + j02 * t02) + dil;
    float s11 = (j11 * t11 + j12 * t12) + dil;
    float s01 = j11 * t01 + j12 * t02;
    float det = s00 * s11 - s01 * s01;
    if (!(det > 0.0f)) return 0;
    ctrx = fx * xz + cx;
    ctry = fy * yz + cy;
    hx = sqrtf(dmax * s00);
    hy = sqrtf(dmax * s11);
    /* det(Sigma') by Cauchy-Binet over the columns t_k = s_k J a_k (a sum of
     * squares: no cancellation for a needle), then the chord through the
     * centre: wch^2 = dmax det / s11 */
    float sk[3] = {sx, sy, sz}, tX[3], tY[3];
    for (int k = 0; k < 3; ++k) {
      tX[k] = sk[k] * (j00 * a[k][0] + j02 * a[k][2]);
      tY[k] = sk[k] * (j11 * a[k][1] + j12 * a[k][2]);
    }
    float m01 = tX[0] * tY[1] - tY[0] * tX[1];
    float m02 = tX[0] * tY[2] - tY[0] * tX[2];
    float m12 = tX[1] * tY[2] - tY[1] * tX[2];
    float x2 = (tX[0] * tX[0] + tX[1] * tX[1]) + tX[2] * tX[2];
    float y2 = (tY[0] * tY[0] + tY[1] * tY[1]) + tY[2] * tY[2];
    float detS = ((m01 * m01 + m02 * m02) + m12 * m12) + (dil * (x2 + y2) + dil * dil);
    kslope = s01 / s11;
    wch = sqrtf((dmax * detS) / s11);
    yoff = (dmax * s01) / hx;
  } else {
    float m0x = sx * a[0][0], m0y = sx * a[0][1], m0z = sx * a[0][2];
    float m1x = sy * a[1][0], m1y = sy * a[1][1], m1z = sy * a[1][2];
    float g2 = m0z * m0z + m1z * m1z;
    float zmin = Z - sqrtf(dmax * g2);
    if (!(zmin > near_z)) {
      whole = 1;
    } else {
      float e0 = m0x - xz * m0z, e1 = m1x - xz * m1z, e2 = X - xz * Z;
      float f0 = m0y - yz * m0z, f1 = m1y - yz * m1z, f2 = Y - yz * Z;
      float D22 = dmax * g2 - Z * Z;
      if (!(D22 < 0.0f)) {
        whole = 1;
      } else {
        float D00 = dmax * (e0 * e0 + e1 * e1) - e2 * e2;
        float D02 = dmax * (e0 * m0z + e1 * m1z) - e2 * Z;
        float D11 = dmax * (f0 * f0 + f1 * f1) - f2 * f2;
        float D12 = dmax * (f0 * m0z + f1 * m1z) - f2 * Z;
        float qx = D02 * D02 - D00 * D22;
        float qy = D12 * D12 - D11 * D22;
        if (!(qx >= 0.0f) || !(qy >= 0.0f)) {
          whole = 1;
        } else {
          float nD = -D22;
          float ox = D02 / D22, oy = D12 / D22;
          ctrx = fx * (xz + ox) + cx;
          ctry = fy * (yz + oy) + cy;
          hx = fx * (sqrtf(qx) / nD);
          hy = fy * (sqrtf(qy) / nD);
          /* the image ellipse's shape from the dual conic D: Sigma_xy =
           * fx fy (D02 D12 - D01 D22) / D22^2 and det Sigma = fx^2 fy^2
           * dmax^2 det(M)^2 / nD^3, M = [e f m_z; ...] the re-centred splat
           * frame (det D = -dmax^2 det(M)^2) */
          float D01 = dmax * (e0 * f0 + e1 * f1) - e2 * f2;
          kslope = (fx * (D02 * D12 - D01 * D22)) / (fy * qy);
          float detM = (e0 * (f1 * Z - f2 * m1z) - e1 * (f0 * Z - f2 * m0z)) + e2 * (f0 * m1z - f1 * m0z);
          wch = ((fx * dmax) * fabsf(detM)) / sqrtf(nD * qy);
          yoff = (kslope * (hy * hy)) / hx;
        }
      }
    }
    if (whole) {
      full = 1;
      disc = 1;
      dP[0] = fx * X + cx * Z; dP[1] = fy * Y + cy * Z; dP[2] = Z;
      dA[0] = fx * m0x + cx * m0z; dA[1] = fy * m0y + cy * m0z; dA[2] = m0z;
      dB[0] = fx * m1x + cx * m1z; dB[1] = fy * m1y + cy * m1z; dB[2] = m1z;
      /* the disc reaches the near plane: a contributing hit lies in the disc
       * (camera-space extents R) at depth in (near, Z + Rz], so x/z and y/z
       * are bounded by the extents divided by the depth bounds */
      float sd = sqrtf(dmax);
      float Rx = sd * sqrtf(m0x * m0x + m1x * m1x);
      float Ry = sd * sqrtf(m0y * m0y + m1y * m1y);
      float zhi = Z + sd * sqrtf(g2);
      float xl = X - Rx, xh = X + Rx, yl = Y - Ry, yh = Y + Ry;
      float nxl = xl >= 0.0f ? xl / zhi : xl / near_z;
      float nxh = xh >= 0.0f ? xh / near_z : xh / zhi;
      float nyl = yl >= 0.0f ? yl / zhi : yl / near_z;
      float nyh = yh >= 0.0f ? yh / near_z : yh / zhi;
      float ilx = fx * nxl + cx, ihx = fx * nxh + cx;
      float ily = fy * nyl + cy, ihy = fy * nyh + cy;
      ctrx = 0.5f * (ilx + ihx);
      ctry = 0.5f * (ily + ihy);
      hx = 0.5f * (ihx - ilx);
      hy = 0.5f * (ihy - ily);
      whole = 0;
    }
  }
  int tx0, tx1, ty0, ty1;
  if (whole) {
    tx0 = 0; tx1 = (W - 1) / tile; ty0 = 0; ty1 = (H - 1) / tile;
    full = 1;
  } else {
    float px = pad_f(hx), py = pad_f(hy);
    if (!c_range(ctrx - px, ctrx + px, W, tile, &tx0, &tx1)) return 0;
    if (!c_range(ctry - py, ctry + py, H, tile, &ty0, &ty1)) return 0;
  }
  rect[0] = tx0; rect[1] = tx1; rect[2] = ty0; rect[3] = ty1;
  /* padded chord parameters: the half chord by pad_f plus 2^-10 hx for the
   * rounding of kslope (y - ctry), the half height by pad_f */
  for (int k = 0; k < ORC_ROWP; ++k) rowp[k] = 0.0f;
  if (disc) {
    int fin = isfinite(dmax);
    for (int k = 0; k < 3; ++k) fin = fin && isfinite(dP[k]) && isfinite(dA[k]) && isfinite(dB[k]);
    if (fin) {
      rowp[0] = dP[0]; rowp[1] = dP[1]; rowp[2] = dP[2]; rowp[3] = dmax;
      rowp[4] = dA[0]; rowp[5] = dA[1]; rowp[6] = dA[2]; rowp[7] = near_z;
      rowp[8] = dB[0]; rowp[9] = dB[1]; rowp[10] = dB[2]; rowp[11] = 2.0f;
    } else {
      rowp[11] = 1.0f;
    }
    return 1;
  }
  float wp = pad_f(wch) + hx * 0x1p-10f, hyp = pad_f(hy), ihy = 1.0f / hyp;
  float yl = ctry - yoff, yr = ctry + yoff;
  if (!(isfinite(kslope) && isfinite(wp) && isfinite(yl) && isfinite(yr) && hyp > 0.0f && isfinite(ihy)))
    full = 1;
  rowp[0] = ctrx; rowp[1] = ctry; rowp[2] = kslope; rowp[3] = wp;
  rowp[4] = ihy; rowp[5] = yl; rowp[6] = yr; rowp[11] = full ? 1.0f : 0.0f;
  return 1;
}

/* The x-range [*xlo, *xhi] of the pixels of tile row ty whose rays hit a
 * disc-mode surfel's disc in front of the near plane.  rowp: the disc's
 * centre C and axes a, b in pixel-homogeneous camera coordinates P = (fx X +
 * cx Z, fy Y + cy Z, Z), its squared radius dmax, near.  A pixel (x, y) sees
 * P(u, v) = C + u a + v b (u^2 + v^2 <= dmax) at x = P0/P2, y = P1/P2 and
 * depth P2; over the row's band of pixel-centre heights [ya, yb] the points
 * seen form the disc cut by three half-planes c + p u + q v >= 0 (P1 - ya P2,
 * yb P2 - P1, P2 - near).  x is a ratio of affine functions, so its extremes
 * over that convex set lie at points of the circle where a plane x P2 = P0
 * touches it, at the lines' crossings with the circle, or at the lines'
 * crossings with each other; every candidate inside the set (with a relative
 * tolerance of 2^-12 on each half-plane and 2^-10 on the radius) is taken.
 * Returns 0 if none is. */
static int disc_span(const float rp[ORC_ROWP], int ty, int tile, float *xlo, float *xhi) {
  const float ya = (float)(ty * tile) + 0.5f, yb = ya + (float)(tile - 1);
  const float CX = rp[0], CY = rp[1], CZ = rp[2], r2 = rp[3];
  const float ax = rp[4], ay = rp[5], az = rp[6], nz = rp[7];
  const float bx = rp[8], by = rp[9], bz = rp[10];
  float c[3], p[3], q[3], tol[3];
  c[0] = CY - ya * CZ; p[0] = ay - ya * az; q[0] = by - ya * bz;
  c[1] = yb * CZ - CY; p[1] = yb * az - ay; q[1] = yb * bz - by;
  c[2] = CZ - nz; p[2] = az; q[2] = bz;
  const float rho = sqrtf(r2);
  for (int k = 0; k < 3; ++k) tol[k] = 0x1p-12f * (fabsf(c[k]) + rho * (fabsf(p[k]) + fabsf(q[k])));
  const float r2t = r2 * 1.0009765625f;
  float cu[11], cv[11];
  int onc[11], nc = 0;
  /* (a) tangency: (CX - x CZ)^2 = r2 ((ax - x az)^2 + (bx - x bz)^2) */
  const float A = CZ * CZ - r2 * (az * az + bz * bz);
  const float B = CX * CZ - r2 * (ax * az + bx * bz);
  const float Cq = CX * CX - r2 * (ax * ax + bx * bx);
  const float dq = B * B - A * Cq;
  if (dq >= 0.0f && A != 0.0f) {
    const float sq = sqrtf(dq);
    float xs[2];
    xs[0] = (B - sq) / A;
    xs[1] = (B + sq) / A;
    for (int k = 0; k < 2; ++k) {
      const float al = CX - xs[k] * CZ, be0 = ax - xs[k] * az, be1 = bx - xs[k] * bz;
      const float bb = be0 * be0 + be1 * be1;
      if (!(bb > 0.0f)) continue;
      const float t = -al / bb;
      cu[nc] = t * be0; cv[nc] = t * be1; onc[nc] = 1; ++nc;
    }
  }
  /* (b) each line's crossings with the circle */
  for (int k = 0; k < 3; ++k) {
    const float pq = p[k] * p[k] + q[k] * q[k];
    if (!(pq > 0.0f)) continue;
    const float t = -c[k] / pq;
    const float fu = t * p[k], fv = t * q[k];
    const float d2 = (c[k] * c[k]) / pq;
    if (!(d2 <= r2t)) continue;
    const float h = sqrtf(fmaxf(r2 - d2, 0.0f) / pq);
    cu[nc] = fu - h * q[k]; cv[nc] = fv + h * p[k]; onc[nc] = 1; ++nc;
    cu[nc] = fu + h * q[k]; cv[nc] = fv - h * p[k]; onc[nc] = 1; ++nc;
  }
  /* (c) the lines' crossings with each other */
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j) {
      const float det = p[i] * q[j] - p[j] * q[i];
      if (det == 0.0f) continue;
      cu[nc] = (q[i] * c[j] - q[j] * c[i]) / det;
      cv[nc] = (p[j] * c[i] - p[i] * c[j]) / det;
      onc[nc] = 0;
      ++nc;
    }
  float lo = INFINITY, hi = -INFINITY;
  for (int k = 0; k < nc; ++k) {
    const float u = cu[k], v = cv[k];
    if (!onc[k] && !(u * u + v * v <= r2t)) continue;
    int ok = 1;
    for (int m = 0; m < 3; ++m)
      if (!((c[m] + p[m] * u) + q[m] * v >= -tol[m])) ok = 0;
    if (!ok) continue;
    const float D = (CZ + az * u) + bz * v;
    if (!(D > 0.0f)) continue;
    const float x = ((CX + ax * u) + bx * v) / D;
    lo = fminf(lo, x);
    hi = fmaxf(hi, x);
  }
  if (!(lo <= hi)) return 0;
  const float pad = 0x1p-9f * fmaxf(fabsf(lo), fabsf(hi)) + 0.0625f;
  *xlo = lo - pad;
  *xhi = hi + pad;
  return 1;
}

/* rowp (ellipse mode, rowp[11] = 0): chord centre x and y, slope, padded half
 * chord, reciprocal of the padded half height, heights of the leftmost and
 * rightmost points; rowp[11] = 1: the whole rectangle; 2: disc mode
 * (disc_span).
 * Tile columns [*c0, *c1] of tile row ty of a binned primitive's tile set:
 * the pixel columns whose centres the padded footprint ellipse reaches in
 * the row's band of pixel-centre heights [ty tile + 0.5, ty tile + tile -
 * 0.5], within the rectangle.  Over the band the chord's left end is least
 * at the band height nearest the ellipse's leftmost point (the left end is
 * convex in y), the right end greatest nearest the rightmost point.  A
 * primitive marked full lists every tile of its rectangle.  Returns 0 if the
 * row lists no tile. */
static int row_span(const float rowp[ORC_ROWP], const int rect[4], int ty, int W, int tile, int *c0, int *c1) {
  if (rowp[11] == 1.0f) {
    *c0 = rect[0];
    *c1 = rect[1];
    return 1;
  }
  if (rowp[11] == 2.0f) {
    float xl, xr;
    int a, b;
    if (!disc_span(rowp, ty, tile, &xl, &xr)) return 0;
    if (!c_range(xl, xr, W, tile, &a, &b)) return 0;
    if (a < rect[0]) a = rect[0];
    if (b > rect[1]) b = rect[1];
    if (a > b) return 0;
    *c0 = a;
    *c1 = b;
    return 1;
  }
  const float cxe = rowp[0], cye = rowp[1], kslope = rowp[2], wp = rowp[3], ihy = rowp[4];
  const float ya = (float)(ty * tile) + 0.5f, yb = ya + (float)(tile - 1);
  const float y1 = fminf(fmaxf(rowp[5], ya), yb), y2 = fminf(fmaxf(rowp[6], ya), yb);
  const float d1 = y1 - cye, d2 = y2 - cye;
  const float t1 = d1 * ihy, t2 = d2 * ihy;
  const float r1 = fmaxf(1.0f - t1 * t1, 0.0f), r2 = fmaxf(1.0f - t2 * t2, 0.0f);
  const float xl = (cxe + kslope * d1) - wp * sqrtf(r1);
  const float xr = (cxe + kslope * d2) + wp * sqrtf(r2);
  int a, b;
  if (!c_range(xl, xr, W, tile, &a, &b)) return 0;
  if (a < rect[0]) a = rect[0];
  if (b > rect[1]) b = rect[1];
  if (a > b) return 0;
  *c0 = a;
  *c1 = b;
  return 1;
}

/* tiles of a binned primitive's tile set */
static int64_t set_count(const float rowp[ORC_ROWP], const int rect[4], int W, int tile) {
  int64_t n = 0;
  for (int ty = rect[2]; ty <= rect[3]; ++ty) {
    int a, b;
    if (row_span(rowp, rect, ty, W, tile, &a, &b)) n += b - a + 1;
  }
  return n;
}

/* cfg32: near, alpha_min, dilation.  rect: n x 4 (tx0,tx1,ty0,ty1), -1 if not
 * binned.  touched: tiles in the primitive's tile set (0 if not binned; a
 * binned primitive whose set is empty is not binned either).  rowp (n x 12,
 * may be NULL): the tile-set parameters. */
void orc_contract_bin(int64_t n, const float *means, const float *log_scales,
                      const float *quats, const float *logits, const uint8_t *types,
                      const float *cam, int W, int H, int tile, const float *cfg32,
                      uint32_t *depth_bits, int32_t *rect, int64_t *touched, float *rowp) {
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    int r[4];
    uint32_t db;
    float rp[ORC_ROWP];
    int ok = contract_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i],
                          types[i], cam, W, H, tile, cfg32[0], cfg32[1], cfg32[2], r, &db, rp);
    depth_bits[i] = db;
    const int64_t cnt = ok ? set_count(rp, r, W, tile) : 0;
    if (cnt > 0) {
      for (int k = 0; k < 4; ++k) rect[4 * i + k] = r[k];
      touched[i] = cnt;
      if (rowp) memcpy(rowp + ORC_ROWP * i, rp, sizeof(rp));
    } else {
      for (int k = 0; k < 4; ++k) rect[4 * i + k] = -1;
      touched[i] = 0;
      if (rowp) memset(rowp + ORC_ROWP * i, 0, sizeof(rp));
    }
  }
}

/* The tile ids of every binned primitive's tile set, row by row and left to
 * right: primitive i's at tiles[first[i] ..], touched[i] of them. */
void orc_contract_tiles(int64_t n, const int32_t *rect, const float *rowp, const int64_t *touched,
                        const int64_t *first, int W, int tile, uint32_t *tiles) {
  const int TX = (W + tile - 1) / tile;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    if (touched[i] <= 0) continue;
    int64_t o = first[i];
    const int *r = rect + 4 * i;
    for (int ty = r[2]; ty <= r[3]; ++ty) {
      int a, b;
      if (!row_span(rowp + ORC_ROWP * i, r, ty, W, tile, &a, &b)) continue;
      for (int tx = a; tx <= b; ++tx) tiles[o++] = (uint32_t)(ty * TX + tx);
    }
  }
}

/* Whether tile (tx, ty) is in the tile set of a binned primitive. */
static int set_has(const float rowp[ORC_ROWP], const int rect[4], int tx, int ty, int W, int tile) {
  if (ty < rect[2] || ty > rect[3] || tx < rect[0] || tx > rect[1]) return 0;
  int a, b;
  return row_span(rowp, rect, ty, W, tile, &a, &b) && tx >= a && tx <= b;
}

float orc_contract_exp(float x) { return orc_c_exp(x); }
float orc_contract_log(float x) { return orc_c_log(x); }

/* ------------------------------------------------------------------------ */
/* (1) FP64 per-pixel renderer                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  int type, valid;
  double alpha;                   /* opacity used for contributions */
  double col[3], nrm[3];
  double X, Y, Z;                 /* camera-space centre */
  uint32_t key;                   /* contract FP32 depth bits: the order key */
  double mx, my, ca, cb, cc;      /* 3D: projected centre, Cholesky factor of the conic */
  double a[3], b[3];              /* 2D: s_x R_cw r0, s_y R_cw r1 */
  double ndot;                    /* |n . mu_c| / |mu_c| */
  double bx0, bx1, by0, by1;      /* padded continuous bbox in pixels */
  int whole;
  int rect[4];                    /* the contract's tile rectangle ... */
  float rowp[ORC_ROWP];           /* ... and tile-set parameters (row_span) */
} prim_t;

typedef struct {
  int64_t n;
  int W, H, deg, nb;
  double R[9], t[3], fx, fy, cx, cy;
  float cam32[16];
  double cfg[CF_COUNT];
  prim_t *P;
  int cell, gx, gy;
  int64_t *cstart;   /* gx*gy+1 */
  int32_t *citems;
  int maxcell;
} orc_ctx;

static void prep_prim(orc_ctx *C, int64_t i, const double *mu64, const double *ls64,
                      const double *q64, double logit64, const double *sh64, int type) {
  prim_t *p = &C->P[i];
  memset(p, 0, sizeof(*p));
  p->type = type;
  const double *Rc = C->R, *tc = C->t;
  const double mu[3] = {mu64[0], mu64[1], mu64[2]};
  const float mu32[3] = {(float)mu64[0], (float)mu64[1], (float)mu64[2]};
  p->X = Rc[0] * mu[0] + Rc[1] * mu[1] + Rc[2] * mu[2] + tc[0];
  p->Y = Rc[3] * mu[0] + Rc[4] * mu[1] + Rc[5] * mu[2] + tc[1];
  p->Z = Rc[6] * mu[0] + Rc[7] * mu[1] + Rc[8] * mu[2] + tc[2];
  {
    /* the order key: binary32 centre depth by the contract's op order */
    const float *R32 = C->cam32, *t32 = C->cam32 + 9;
    float Z32 = ((R32[6] * mu32[0] + R32[7] * mu32[1]) + R32[8] * mu32[2]) + t32[2];
    p->key = bits_from_f32(Z32);
  }
  const double nearz = C->cfg[CF_NEAR], amin = C->cfg[CF_ALPHA_MIN];
  {
    /* visibility is the binning contract's binary32 decision: a primitive the
     * contract does not bin (behind the near plane, below alpha_min, a
     * degenerate projection, or parameters that overflow binary32) is not
     * rendered */
    const float ls32[3] = {(float)ls64[0], (float)ls64[1], (float)ls64[2]};
    const float q32[4] = {(float)q64[0], (float)q64[1], (float)q64[2], (float)q64[3]};
    uint32_t dbb;
    if (!contract_one(mu32, ls32, q32, (float)logit64, type, C->cam32, C->W, C->H, 16,
                      (float)nearz, (float)amin, (float)C->cfg[CF_DILATION], p->rect, &dbb, p->rowp))
      return;
    if (set_count(p->rowp, p->rect, C->W, 16) == 0) return;
  }
  /* (the contract's binary32 centre depth is beyond the near plane; the FP64
   * depth may differ from it by a rounding, which changes nothing below) */
  /* activations (Sec. 3.1): scale = exp(log s), unit quaternion, sigmoid */
  double s[3] = {exp(ls64[0]), exp(ls64[1]), exp(ls64[2])};
  double q[4] = {q64[0], q64[1], q64[2], q64[3]};
  double qn = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  if (!(qn > 0)) return;
  double Rq[9];
  quat_to_rot(q, Rq);
  double alpha = 1.0 / (1.0 + exp(-logit64));
  double alpha_bb = alpha;
  if (type == 0) {
    /* scale modulation for 2D Gaussians (Eqs. 6-7) */
    double sz = s[2];
    double g = 1.0 / (1.0 + exp(-(sz - C->cfg[CF_THETA_Z]) / C->cfg[CF_T_Z]));
    alpha *= exp(-C->cfg[CF_LAMBDA_Z] * (g * sz));
  }
  p->alpha = alpha;
  if (!(alpha_bb >= amin * (1.0 - AMB_ALPHA_REL))) return;
  /* camera-space axes a_k = R_cw r_k */
  double ax[3][3];
  for (int k = 0; k < 3; ++k)
    for (int r = 0; r < 3; ++r)
      ax[k][r] = Rc[3 * r] * Rq[k] + Rc[3 * r + 1] * Rq[3 + k] + Rc[3 * r + 2] * Rq[6 + k];
  /* normal: axis of the smallest scale (2D: the z axis), facing the camera */
  int kn;
  if (type == 0) kn = 2;
  else if (ls64[2] <= ls64[0] && ls64[2] <= ls64[1]) kn = 2;
  else if (ls64[0] <= ls64[1]) kn = 0;
  else kn = 1;
  double nd = ax[kn][0] * p->X + ax[kn][1] * p->Y + ax[kn][2] * p->Z;
  double sg = nd > 0 ? -1.0 : 1.0;
  for (int r = 0; r < 3; ++r) p->nrm[r] = sg * ax[kn][r];
  double mun = sqrt(p->X * p->X + p->Y * p->Y + p->Z * p->Z);
  p->ndot = fabs(nd) / mun;
  /* colour from SH (Sec. 3.1), view direction from the camera centre */
  {
    double cc[3];
    for (int r = 0; r < 3; ++r)
      cc[r] = -(C->R[0 + r] * tc[0] + C->R[3 + r] * tc[1] + C->R[6 + r] * tc[2]);
    double dv[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
    double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double Yb[16];
    sh_basis(C->deg, dv[0] / dn, dv[1] / dn, dv[2] / dn, Yb);
    for (int ch = 0; ch < 3; ++ch) {
      double v = 0.5;
      for (int k = 0; k < C->nb; ++k) v += sh64[3 * k + ch] * Yb[k];
      p->col[ch] = v > 0 ? v : 0;
    }
  }
  double dmax = 2.0 * log(alpha_bb / amin);
  if (dmax < 0) dmax = 0;
  dmax += 1e-3; /* the bbox is an index only: generous */
  const double fx = C->fx, fy = C->fy, cx = C->cx, cy = C->cy;
  double X = p->X, Y = p->Y, Z = p->Z;
  if (type == 1) {
    /* EWA projection, App. C Eq. 13: Sigma' = J W Sigma W^T J^T = T T^T with
     * T = J W R S (2x3).  det Sigma' by Cauchy-Binet (sum of squared 2x2
     * minors of T) and Eq. 1's quadratic form through the Cholesky factor of
     * Sigma'^-1, so needle-like footprints keep full precision. */
    double J[2][3] = {{fx / Z, 0, -fx * X / (Z * Z)}, {0, fy / Z, -fy * Y / (Z * Z)}};
    double T[2][3];
    for (int r = 0; r < 2; ++r)
      for (int k = 0; k < 3; ++k)
        T[r][k] = s[k] * (J[r][0] * ax[k][0] + J[r][1] * ax[k][1] + J[r][2] * ax[k][2]);
    double S2[2][2];
    for (int r = 0; r < 2; ++r)
      for (int c2 = 0; c2 < 2; ++c2)
        S2[r][c2] = T[r][0] * T[c2][0] + T[r][1] * T[c2][1] + T[r][2] * T[c2][2];
    const double dil = C->cfg[CF_DILATION];
    double m01 = T[0][0] * T[1][1] - T[1][0] * T[0][1];
    double m02 = T[0][0] * T[1][2] - T[1][0] * T[0][2];
    double m12 = T[0][1] * T[1][2] - T[1][1] * T[0][2];
    double det = m01 * m01 + m02 * m02 + m12 * m12 + dil * (S2[0][0] + S2[1][1]) + dil * dil;
    S2[0][0] += dil;
    S2[1][1] += dil;
    if (!(det > 0) || !(S2[1][1] > 0)) return;
    p->ca = sqrt(S2[1][1] / det);              /* W00 */
    p->cb = -S2[0][1] / sqrt(S2[1][1] * det);   /* W01 */
    p->cc = 1.0 / sqrt(S2[1][1]);               /* W11 */
    p->mx = fx * X / Z + cx;
    p->my = fy * Y / Z + cy;
    double hx = sqrt(dmax * S2[0][0]), hy = sqrt(dmax * S2[1][1]);
    hx = hx * 1.01 + 2.0;
    hy = hy * 1.01 + 2.0;
    p->bx0 = p->mx - hx; p->bx1 = p->mx + hx;
    p->by0 = p->my - hy; p->by1 = p->my + hy;
  } else {
    p->mx = fx * X / Z + cx;
    p->my = fy * Y / Z + cy;
    for (int r = 0; r < 3; ++r) { p->a[r] = s[0] * ax[0][r]; p->b[r] = s[1] * ax[1][r]; }
    /* bbox of the image of the disc u^2+v^2 <= dmax: whole image unless the
     * disc lies entirely in front of the camera */
    double g2 = p->a[2] * p->a[2] + p->b[2] * p->b[2];
    double zmin = Z - sqrt(dmax * g2);
    if (!(zmin > 0.5 * nearz)) {
      p->whole = 1;
    } else {
      /* conic of the disc image, via the dual conic in normalised coords */
      double xz = X / Z, yz = Y / Z;
      double e0 = p->a[0] - xz * p->a[2], e1 = p->b[0] - xz * p->b[2], e2 = X - xz * Z;
      double f0 = p->a[1] - yz * p->a[2], f1 = p->b[1] - yz * p->b[2], f2 = Y - yz * Z;
      double D22 = dmax * g2 - Z * Z;
      double D00 = dmax * (e0 * e0 + e1 * e1) - e2 * e2;
      double D02 = dmax * (e0 * p->a[2] + e1 * p->b[2]) - e2 * Z;
      double D11 = dmax * (f0 * f0 + f1 * f1) - f2 * f2;
      double D12 = dmax * (f0 * p->a[2] + f1 * p->b[2]) - f2 * Z;
      double qx = D02 * D02 - D00 * D22, qy = D12 * D12 - D11 * D22;
      if (!(D22 < 0) || qx < 0 || qy < 0) {
        p->whole = 1;
      } else {
        double ctx = fx * (xz + D02 / D22) + cx, cty = fy * (yz + D12 / D22) + cy;
        double hx = fx * sqrt(qx) / (-D22), hy = fy * sqrt(qy) / (-D22);
        hx = hx * 1.01 + 2.0;
        hy = hy * 1.01 + 2.0;
        p->bx0 = ctx - hx; p->bx1 = ctx + hx;
        p->by0 = cty - hy; p->by1 = cty + hy;
      }
    }
  }
  p->valid = 1;
}

static void build_grid(orc_ctx *C) {
  int cell = C->cell;
  C->gx = (C->W + cell - 1) / cell;
  C->gy = (C->H + cell - 1) / cell;
  int64_t ncell = (int64_t)C->gx * C->gy;
  int64_t *cnt = (int64_t *)calloc(ncell + 1, sizeof(int64_t));
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      int64_t acc = 0;
      for (int64_t c = 0; c < ncell; ++c) { int64_t v = cnt[c]; C->cstart[c] = acc; acc += v; cnt[c] = 0; }
      C->cstart[ncell] = acc;
      C->citems = (int32_t *)malloc(sizeof(int32_t) * (acc > 0 ? acc : 1));
    }
    for (int64_t i = 0; i < C->n; ++i) {
      prim_t *p = &C->P[i];
      if (!p->valid) continue;
      int x0, x1, y0, y1;
      if (p->whole) {
        x0 = 0; x1 = C->gx - 1; y0 = 0; y1 = C->gy - 1;
      } else {
        double lx = floor(p->bx0 / cell), hx = floor(p->bx1 / cell);
        double ly = floor(p->by0 / cell), hy = floor(p->by1 / cell);
        if (hx < 0 || hy < 0 || lx > C->gx - 1 || ly > C->gy - 1) continue;
        x0 = lx < 0 ? 0 : (int)lx; x1 = hx > C->gx - 1 ? C->gx - 1 : (int)hx;
        y0 = ly < 0 ? 0 : (int)ly; y1 = hy > C->gy - 1 ? C->gy - 1 : (int)hy;
      }
      for (int yy = y0; yy <= y1; ++yy)
        for (int xx = x0; xx <= x1; ++xx) {
          int64_t c = (int64_t)yy * C->gx + xx;
          if (pass == 0) cnt[c]++;
          else C->citems[C->cstart[c] + cnt[c]++] = (int32_t)i;
        }
    }
  }
  int maxc = 0;
  for (int64_t c = 0; c < ncell; ++c) {
    int64_t v = C->cstart[c + 1] - C->cstart[c];
    if (v > maxc) maxc = (int)v;
  }
  C->maxcell = maxc;
  free(cnt);
}

/* Parameters are double arrays (float32 inputs widen exactly); the order key
 * is the contract's binary32 depth of the mean rounded to binary32.
 * cam: float32 R[9] t[3] fx fy cx cy; cfg: double[CF_COUNT]. */
void *orc_prepare(int64_t n, const double *means, const double *log_scales, const double *quats,
                  const double *logits, const double *sh, const uint8_t *types, int sh_deg,
                  const float *cam, int W, int H, const double *cfg) {
  orc_ctx *C = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  C->n = n; C->W = W; C->H = H; C->deg = sh_deg; C->nb = (sh_deg + 1) * (sh_deg + 1);
  for (int k = 0; k < 9; ++k) C->R[k] = cam[k];
  for (int k = 0; k < 3; ++k) C->t[k] = cam[9 + k];
  C->fx = cam[12]; C->fy = cam[13]; C->cx = cam[14]; C->cy = cam[15];
  memcpy(C->cam32, cam, sizeof(float) * 16);
  memcpy(C->cfg, cfg, sizeof(double) * CF_COUNT);
  C->P = (prim_t *)malloc(sizeof(prim_t) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    prep_prim(C, i, means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i],
              sh + (int64_t)3 * C->nb * i, types[i]);
  C->cell = 32;
  C->cstart = (int64_t *)malloc(sizeof(int64_t) * ((int64_t)((W + 31) / 32) * ((H + 31) / 32) + 1));
  build_grid(C);
  return C;
}

/* Re-derive primitive i from new parameters (finite differences).  The grid
 * is not rebuilt: the bbox padding covers perturbations of ~1e-4 px. */
void orc_set_prim(void *ctx, int64_t i, const double *mean, const double *ls, const double *q,
                  double logit, const double *sh, int type) {
  orc_ctx *C = (orc_ctx *)ctx;
  prep_prim(C, i, mean, ls, q, logit, sh, type);
}

void orc_free(void *ctx) {
  orc_ctx *C = (orc_ctx *)ctx;
  if (!C) return;
  free(C->P); free(C->cstart); free(C->citems); free(C);
}

/* a listed (pixel, primitive) pair */
enum { PA_ALPHA = 1, PA_NEAR = 2, PA_FLIP = 4 };
typedef struct {
  uint32_t key;
  int32_t id;
  uint8_t flags;        /* PA_*: which of its decisions sit in a band */
  uint8_t a_ok, z_ok;   /* the FP64 outcomes: ag >= alpha_min, hit beyond near */
  double ag;            /* alpha exp(-d/2), unclamped */
  double dag;           /* conditioning bound on the binary32 error of ag */
  double z;             /* per-pixel depth: centre depth (3D), hit depth (2D) */
} contrib_t;

static int cmp_contrib(const void *A, const void *B) {
  const contrib_t *a = (const contrib_t *)A, *b = (const contrib_t *)B;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->id < b->id ? -1 : (a->id > b->id);
}

/* ray-splat intersection (App. C): solve mu_c + u a + v b = tau ray(px, py)
 * by Gaussian elimination with partial pivoting.  Returns 0 if the system is
 * singular (the ray lies in the splat's plane). */
static int surfel_hit(const orc_ctx *C, const prim_t *p, double px, double py, double sol[3]) {
  double ray[3] = {(px - C->cx) / C->fx, (py - C->cy) / C->fy, 1.0};
  double A[3][4] = {{p->a[0], p->b[0], -ray[0], -p->X},
                    {p->a[1], p->b[1], -ray[1], -p->Y},
                    {p->a[2], p->b[2], -ray[2], -p->Z}};
  double scale = sqrt(p->a[0] * p->a[0] + p->a[1] * p->a[1] + p->a[2] * p->a[2]) *
                 sqrt(p->b[0] * p->b[0] + p->b[1] * p->b[1] + p->b[2] * p->b[2]) *
                 sqrt(ray[0] * ray[0] + ray[1] * ray[1] + 1.0);
  double detv = 1.0;
  for (int c = 0; c < 3; ++c) {
    int piv = c;
    for (int r = c + 1; r < 3; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < 4; ++k) { double tmp = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = tmp; }
      detv = -detv;
    }
    detv *= A[c][c];
    if (A[c][c] == 0.0) return 0;
    for (int r = c + 1; r < 3; ++r) {
      double f = A[r][c] / A[c][c];
      for (int k = c; k < 4; ++k) A[r][k] -= f * A[c][k];
    }
  }
  if (fabs(detv) <= 1e-12 * scale) return 0;
  for (int r = 2; r >= 0; --r) {
    double v = A[r][3];
    for (int k = r + 1; k < 3; ++k) v -= A[r][k] * sol[k];
    sol[r] = v / A[r][r];
  }
  return 1;
}

/* Conditioning of a pair's splat-frame coordinates (u, v) at the pixel
 * centre (px, py): a binary32 evaluation from the offset (ex, ey) to the
 * projected centre, u = du/dx ex + du/dy ey (likewise v), carries up to
 * COND_ULPS ulps of the cancelling terms |du/dx ex| + |du/dy ey|; *du and *dv
 * are those bounds.  A surfel's derivatives are taken by differences of the
 * ray-splat solve 1e-3 px apart. */
static void cond_uv(const orc_ctx *C, const prim_t *p, double px, double py, double u, double v, double *du,
                    double *dv) {
  double ex = px - p->mx, ey = py - p->my, dux, duy, dvx, dvy;
  if (p->type == 1) {
    dux = p->ca; duy = p->cb; dvx = 0.0; dvy = p->cc;
  } else {
    double s1[3], s2[3];
    const double hh = 1e-3;
    if (surfel_hit(C, p, px + hh, py, s1) && surfel_hit(C, p, px, py + hh, s2)) {
      dux = (s1[0] - u) / hh; dvx = (s1[1] - v) / hh;
      duy = (s2[0] - u) / hh; dvy = (s2[1] - v) / hh;
    } else {
      dux = duy = dvx = dvy = 0.0;
    }
  }
  const double eps32 = 5.960464477539063e-08;
  *du = COND_ULPS * eps32 * (fabs(dux * ex) + fabs(duy * ey));
  *dv = COND_ULPS * eps32 * (fabs(dvx * ex) + fabs(dvy * ey));
}

/* Unified distance (Eq. 1) and contribution (Sec. 3.1) of primitive p at the
 * pixel centre (px, py).  Returns 1 and fills *c if the pair must be listed:
 * it contributes, or one of its decisions sits in a band (c->flags).  The
 * blend decides whether a listed pair matters: only pairs reached before the
 * pixel terminates can change the result. */
static int eval_pair(const orc_ctx *C, const prim_t *p, double px, double py, contrib_t *c) {
  double d, z, u, v;
  const double amin = C->cfg[CF_ALPHA_MIN], nearz = C->cfg[CF_NEAR];
  uint8_t flags = 0;
  int z_ok = 1;
  if (p->type == 1) {
    double dx = px - p->mx, dy = py - p->my;
    u = p->ca * dx + p->cb * dy;
    v = p->cc * dy;
    d = u * u + v * v;
    z = p->Z;
  } else {
    double sol[3];
    if (!surfel_hit(C, p, px, py, sol)) return 0;
    u = sol[0];
    v = sol[1];
    z = sol[2];
    d = u * u + v * v;
    z_ok = z > nearz;
    if (fabs(z - nearz) <= AMB_NEAR_REL * fmax(1.0, nearz)) flags |= PA_NEAR;
  }
  const double ag = p->alpha * exp(-0.5 * d);
  if (ag < 0.1 * amin && !(flags & PA_NEAR)) return 0;  /* no binary32 error reaches the threshold from here */
  /* conditioning of (u, v) as functions of the offset to the centre */
  double du, dv;
  cond_uv(C, p, px, py, u, v, &du, &dv);
  const double dd = 2.0 * (fabs(u) * du + fabs(v) * dv) + du * du + dv * dv;
  /* ag moves by at most ag (e^(dd/2) - 1) when d moves by dd */
  const double dag = ag * expm1(0.5 * dd);
  const int a_ok = ag >= amin;
  if (fabs(ag - amin) <= fmax(AMB_ALPHA_REL * amin, dag)) flags |= PA_ALPHA;
  if (p->ndot < AMB_FLIP) flags |= PA_FLIP;
  if (!(a_ok && z_ok) && !(flags & (PA_ALPHA | PA_NEAR))) return 0;
  c->flags = flags;
  c->a_ok = (uint8_t)a_ok;
  c->z_ok = (uint8_t)z_ok;
  c->ag = ag;
  c->dag = dag;
  c->z = z;
  return 1;
}

/* One blend of a pixel's sorted pairs (Eq. 2, front to back) with the
 * outcome of the j-th ambiguous decision met taken from bit j of `choice`
 * (0: the FP64 outcome, 1: the other one).  o: r, g, b, depth, nx, ny, nz,
 * alpha, T_final, contributors; tol: per-output bound of the conditioning
 * errors (dag) and of the faint decisions carried through Eq. 2, and in
 * tol[9] the number of faint decisions (the contributor count's slack).
 * Returns the number of ambiguous decisions met. */
static int blend_run(const orc_ctx *C, const contrib_t *buf, int cnt, uint32_t choice, const double vmax[10],
                     double o[10], double tol[10], int *loose) {
  const double Tmin = C->cfg[CF_T_MIN], amax = C->cfg[CF_ALPHA_MAX];
  double T = 1.0, Cc[3] = {0, 0, 0}, D = 0, Nn[3] = {0, 0, 0}, tT = 0.0;
  int used = 0, nd = 0;
  *loose = 0;
  for (int k = 0; k < 10; ++k) tol[k] = 0.0;
#define TAKE_BIT() (nd < 32 ? (int)((choice >> nd++) & 1u) : (nd++, 0))
  for (int k = 0; k < cnt; ++k) {
    const contrib_t *c = &buf[k];
    const prim_t *p = &C->P[c->id];
    int a_ok = c->a_ok, z_ok = c->z_ok;
    if (c->flags & PA_ALPHA) {
      const double wmax = (c->ag < amax ? c->ag : amax) * T;
      if (wmax <= ORC_FAINT && !(c->flags & PA_NEAR)) {
        const double v[9] = {p->col[0], p->col[1], p->col[2], c->z, p->nrm[0], p->nrm[1], p->nrm[2], 1.0, 1.0};
        for (int ch = 0; ch < 9; ++ch) tol[ch] += wmax * (fabs(v[ch]) + vmax[ch]);
        tol[9] += 1.0;
        tT += wmax;
      } else {
        a_ok ^= TAKE_BIT();
      }
    }
    if (c->flags & PA_NEAR) z_ok ^= TAKE_BIT();
    if (!(a_ok && z_ok)) continue;
    const double at = c->ag < amax ? c->ag : amax;
    const double Tn = T * (1.0 - at);
    int stop = Tn < Tmin;
    const double band = fmax(AMB_T_REL * Tmin, tT);
    if (fabs(Tn - Tmin) <= band) {
      if (band > 0.5 * Tmin) {
        /* the conditioning errors make the binary32 transmittance too
         * uncertain to place the stop: stopping here or at any later pair
         * moves each output by at most T (|v| + max |v|), since everything
         * blended from here on weighs at most T; added once, and the
         * contributor count is left unchecked */
        if (!*loose)
          for (int ch = 0; ch < 9; ++ch) tol[ch] += T * 2.0 * vmax[ch];
        *loose = 1;
        tol[9] = 1e9;
      } else {
        stop ^= TAKE_BIT();
      }
    }
    if (stop) break;
    double sg = 1.0;
    if (c->flags & PA_FLIP) sg = TAKE_BIT() ? -1.0 : 1.0;
    const double w = at * T;
    for (int r = 0; r < 3; ++r) { Cc[r] += w * p->col[r]; Nn[r] += w * sg * p->nrm[r]; }
    D += w * c->z;
    /* conditioning: moving this contribution by dat moves output ch by at
     * most dat T (|v_ch| + max |v| over the pixel's pairs and background) */
    const double dat = (c->ag - c->dag > amax) ? 0.0 : c->dag;
    if (dat > 0.0) {
      const double v[10] = {p->col[0], p->col[1], p->col[2], c->z, p->nrm[0], p->nrm[1], p->nrm[2], 1.0, 1.0, 0.0};
      for (int ch = 0; ch < 9; ++ch) tol[ch] += dat * T * (fabs(v[ch]) + vmax[ch]);
      tT += dat * T;
    }
    T = Tn;
    used++;
  }
#undef TAKE_BIT
  o[0] = Cc[0] + T * C->cfg[CF_BG0];
  o[1] = Cc[1] + T * C->cfg[CF_BG1];
  o[2] = Cc[2] + T * C->cfg[CF_BG2];
  o[3] = D;
  o[4] = Nn[0]; o[5] = Nn[1]; o[6] = Nn[2];
  o[7] = 1.0 - T;
  o[8] = T;
  o[9] = used;
  return nd;
}

/* Every outcome of the ambiguous decisions, depth first: a run that meets a
 * decision beyond its fixed prefix splits there.  leaves: up to ORC_MAXV x 20
 * doubles (o[10], tol[10]).  Sets *over (and stops) when the results would
 * exceed ORC_MAXV or a path meets more than ORC_MAXDEC decisions. */
static void enum_leaves(const orc_ctx *C, const contrib_t *buf, int cnt, uint32_t prefix, int plen,
                        const double vmax[10], double *leaves, int *nleaves, int *over) {
  if (*over) return;
  double o[10], tol[10];
  int loose;
  const int nd = blend_run(C, buf, cnt, prefix, vmax, o, tol, &loose);
  if (nd <= plen) {
    if (*nleaves == ORC_MAXV) {
      *over = 1;
      return;
    }
    double *L = leaves + 20 * (*nleaves);
    for (int k = 0; k < 10; ++k) { L[k] = o[k]; L[10 + k] = tol[k]; }
    (*nleaves)++;
    return;
  }
  if (plen == ORC_MAXDEC) {
    *over = 1;
    return;
  }
  enum_leaves(C, buf, cnt, prefix, plen + 1, vmax, leaves, nleaves, over);
  enum_leaves(C, buf, cnt, prefix | (1u << plen), plen + 1, vmax, leaves, nleaves, over);
}

/* The sorted pairs of pixel (ix, iy) and the per-output magnitudes bounding
 * what lies behind a pair (for the conditioning tolerance). */
static int pixel_pairs(const orc_ctx *C, int ix, int iy, contrib_t *buf, double vmax[10], int64_t skip) {
  double px = ix + 0.5, py = iy + 0.5;
  int cxi = ix / C->cell, cyi = iy / C->cell;
  int64_t c = (int64_t)cyi * C->gx + cxi;
  int cnt = 0;
  for (int k = 0; k < 10; ++k) vmax[k] = 0.0;
  for (int r = 0; r < 3; ++r) vmax[r] = fabs(C->cfg[CF_BG0 + r]);
  vmax[7] = vmax[8] = 1.0;
  for (int64_t k = C->cstart[c]; k < C->cstart[c + 1]; ++k) {
    int32_t id = C->citems[k];
    const prim_t *p = &C->P[id];
    if (!p->valid || id == skip) continue;
    /* a pair is evaluated only in the tiles of the primitive's tile set */
    if (!set_has(p->rowp, p->rect, ix / 16, iy / 16, C->W, 16)) continue;
    if (eval_pair(C, p, px, py, &buf[cnt])) {
      buf[cnt].key = p->key;
      buf[cnt].id = id;
      const double v[7] = {p->col[0], p->col[1], p->col[2], buf[cnt].z, p->nrm[0], p->nrm[1], p->nrm[2]};
      for (int ch = 0; ch < 7; ++ch)
        if (fabs(v[ch]) > vmax[ch]) vmax[ch] = fabs(v[ch]);
      cnt++;
    }
  }
  qsort(buf, cnt, sizeof(contrib_t), cmp_contrib);
  return cnt;
}

/* Render npix pixels (pix: npix x 2 int32 pixel indices, or NULL = full frame
 * in row-major order), taking every decision the FP64 way.
 * out: npix x 10 doubles [r, g, b, depth, nx, ny, nz, alpha, T_final,
 * n_contrib].  flags (npix): bit 0 = ambiguous decisions met (more results
 * are correct: orc_render_variants lists them), bit 1 = more correct results
 * than the renderer enumerates (ORC_MAXV), or more than ORC_MAXDEC decisions
 * on one path (not comparable), bit 2 = the conditioning errors leave the
 * stop point unplaceable (its effect is in the tolerance, the contributor
 * count unchecked).  tol (npix x 10, may be NULL): the tolerance of this
 * result (tol[9]: the contributor count's slack). */
void orc_render(void *ctx, int64_t npix, const int32_t *pix, double *out, uint8_t *flags, double *tol) {
  orc_ctx *C = (orc_ctx *)ctx;
  if (!pix) npix = (int64_t)C->W * C->H;
#pragma omp parallel
  {
    contrib_t *buf = (contrib_t *)malloc(sizeof(contrib_t) * (C->maxcell > 0 ? C->maxcell : 1));
    double *lv = (double *)malloc(sizeof(double) * ORC_MAXV * 20);
#pragma omp for schedule(dynamic, 64)
    for (int64_t q = 0; q < npix; ++q) {
      int ix, iy;
      if (pix) { ix = pix[2 * q]; iy = pix[2 * q + 1]; }
      else { ix = (int)(q % C->W); iy = (int)(q / C->W); }
      double vmax[10], t[10];
      int loose;
      const int cnt = pixel_pairs(C, ix, iy, buf, vmax, -1);
      const int nd = blend_run(C, buf, cnt, 0u, vmax, out + 10 * q, t, &loose);
      uint8_t f = loose ? 4 : 0;
      if (nd > 0) f |= 1;
      if (nd > ORC_MAXDEC) f |= 2;
      else if (nd > 0) {
        /* a branch can meet decisions the FP64 path does not */
        int nl = 0, over = 0;
        enum_leaves(C, buf, cnt, 0u, 0, vmax, lv, &nl, &over);
        if (over) f |= 2;
      }
      flags[q] = f;
      if (tol)
        for (int k = 0; k < 10; ++k) tol[10 * q + k] = t[k];
    }
    free(buf);
    free(lv);
  }
}

/* Every correct result of npix pixels: nvar[q] results (1 .. ORC_MAXV) of 20
 * doubles each in leaves[q * ORC_MAXV * 20 ..]: the 10 outputs of orc_render
 * and their conditioning tolerance.  The first is orc_render's. */
void orc_render_variants(void *ctx, int64_t npix, const int32_t *pix, int32_t *nvar, double *leaves) {
  orc_ctx *C = (orc_ctx *)ctx;
#pragma omp parallel
  {
    contrib_t *buf = (contrib_t *)malloc(sizeof(contrib_t) * (C->maxcell > 0 ? C->maxcell : 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < npix; ++q) {
      double vmax[10];
      const int cnt = pixel_pairs(C, pix[2 * q], pix[2 * q + 1], buf, vmax, -1);
      int nl = 0, over = 0;
      enum_leaves(C, buf, cnt, 0u, 0, vmax, leaves + (int64_t)q * ORC_MAXV * 20, &nl, &over);
      nvar[q] = nl;
    }
    free(buf);
  }
}

int orc_max_variants(void) { return ORC_MAXV; }

/* The primitives whose pairs Eq. 2 blends at each of npix pixels (every
 * decision the FP64 way), front to back: ids[q * maxc ..], at most maxc per
 * pixel, count[q] of them.  Used to choose the primitives a finite-difference
 * check looks at, among those an image shows. */
void orc_pixel_contributors(void *ctx, int64_t npix, const int32_t *pix, int maxc, int32_t *ids, int32_t *count) {
  orc_ctx *C = (orc_ctx *)ctx;
  const double Tmin = C->cfg[CF_T_MIN], amax = C->cfg[CF_ALPHA_MAX];
#pragma omp parallel
  {
    contrib_t *buf = (contrib_t *)malloc(sizeof(contrib_t) * (C->maxcell > 0 ? C->maxcell : 1));
#pragma omp for schedule(dynamic, 4)
    for (int64_t q = 0; q < npix; ++q) {
      double vmax[10];
      const int cnt = pixel_pairs(C, pix[2 * q], pix[2 * q + 1], buf, vmax, -1);
      double T = 1.0;
      int n = 0;
      for (int k = 0; k < cnt; ++k) {
        if (!(buf[k].a_ok && buf[k].z_ok)) continue;
        const double at = buf[k].ag < amax ? buf[k].ag : amax;
        const double Tn = T * (1.0 - at);
        if (Tn < Tmin) break;
        if (n < maxc) ids[q * maxc + n] = buf[k].id;
        n++;
        T = Tn;
      }
      count[q] = n < maxc ? n : maxc;
    }
    free(buf);
  }
}

/* Finite differences of one primitive.  A central difference changes only
 * primitive i, so the pairs of every other primitive at the pixels looked at
 * are evaluated and sorted once (orc_fd_begin); each orc_fd_render then
 * evaluates primitive i with its current parameters (orc_set_prim), inserts
 * its pair in the sorted order and blends: the same pairs, order and Eq. 2
 * as orc_render, at a fraction of the cost. */
typedef struct {
  int64_t i, npix;
  int32_t *pix;
  contrib_t **list;
  int *cnt;
  double *vmax;
} orc_fd_t;

void *orc_fd_begin(void *ctx, int64_t i, int64_t npix, const int32_t *pix) {
  orc_ctx *C = (orc_ctx *)ctx;
  orc_fd_t *F = (orc_fd_t *)calloc(1, sizeof(orc_fd_t));
  F->i = i;
  F->npix = npix;
  F->pix = (int32_t *)malloc(sizeof(int32_t) * 2 * (npix > 0 ? npix : 1));
  memcpy(F->pix, pix, sizeof(int32_t) * 2 * npix);
  F->list = (contrib_t **)calloc(npix > 0 ? npix : 1, sizeof(contrib_t *));
  F->cnt = (int *)calloc(npix > 0 ? npix : 1, sizeof(int));
  F->vmax = (double *)calloc(10 * (npix > 0 ? npix : 1), sizeof(double));
#pragma omp parallel
  {
    contrib_t *buf = (contrib_t *)malloc(sizeof(contrib_t) * (C->maxcell > 0 ? C->maxcell : 1));
#pragma omp for schedule(dynamic, 1)
    for (int64_t q = 0; q < npix; ++q) {
      const int cnt = pixel_pairs(C, pix[2 * q], pix[2 * q + 1], buf, F->vmax + 10 * q, i);
      F->list[q] = (contrib_t *)malloc(sizeof(contrib_t) * (cnt + 1));
      memcpy(F->list[q], buf, sizeof(contrib_t) * cnt);
      F->cnt[q] = cnt;
    }
    free(buf);
  }
  return F;
}

/* out: npix x 10 as orc_render (every decision the FP64 way); flags: bit 0
 * if an ambiguous decision was met (the difference is then not a
 * derivative), bit 2 as orc_render; tol (may be NULL): as orc_render; pos
 * (may be NULL): primitive i's place in the pixel's sorted pairs, -1 if not
 * listed (a change between two parameter values means the blend order
 * changed, so the difference is not a derivative either). */
void orc_fd_render(void *ctx, void *fd, double *out, uint8_t *flags, double *tol, int32_t *pos) {
  orc_ctx *C = (orc_ctx *)ctx;
  orc_fd_t *F = (orc_fd_t *)fd;
  const prim_t *p = &C->P[F->i];
#pragma omp parallel
  {
    contrib_t *buf = (contrib_t *)malloc(sizeof(contrib_t) * (C->maxcell + 1));
#pragma omp for schedule(static)
    for (int64_t q = 0; q < F->npix; ++q) {
      const int n0 = F->cnt[q];
      double vmax[10];
      memcpy(vmax, F->vmax + 10 * q, sizeof(vmax));
      int cnt = 0;
      contrib_t c;
      memset(&c, 0, sizeof(c));
      const int listed = p->valid && set_has(p->rowp, p->rect, F->pix[2 * q] / 16, F->pix[2 * q + 1] / 16, C->W, 16) &&
                         eval_pair(C, p, F->pix[2 * q] + 0.5, F->pix[2 * q + 1] + 0.5, &c);
      if (listed) {
        c.key = p->key;
        c.id = (int32_t)F->i;
        const double v[7] = {p->col[0], p->col[1], p->col[2], c.z, p->nrm[0], p->nrm[1], p->nrm[2]};
        for (int ch = 0; ch < 7; ++ch)
          if (fabs(v[ch]) > vmax[ch]) vmax[ch] = fabs(v[ch]);
      }
      /* merge primitive i's pair into the sorted list */
      int placed = !listed, at = -1;
      for (int k = 0; k < n0; ++k) {
        if (!placed && cmp_contrib(&c, &F->list[q][k]) < 0) {
          at = cnt;
          buf[cnt++] = c;
          placed = 1;
        }
        buf[cnt++] = F->list[q][k];
      }
      if (!placed) {
        at = cnt;
        buf[cnt++] = c;
      }
      if (pos) pos[q] = at;
      double t[10];
      int loose;
      const int nd = blend_run(C, buf, cnt, 0u, vmax, out + 10 * q, t, &loose);
      flags[q] = (uint8_t)((nd > 0 ? 1 : 0) | (loose ? 4 : 0));
      if (tol)
        for (int k = 0; k < 10; ++k) tol[10 * q + k] = t[k];
    }
    free(buf);
  }
}

void orc_fd_end(void *fd) {
  orc_fd_t *F = (orc_fd_t *)fd;
  if (!F) return;
  for (int64_t q = 0; q < F->npix; ++q) free(F->list[q]);
  free(F->list); free(F->cnt); free(F->vmax); free(F->pix); free(F);
}

/* The contribution alpha exp(-d/2) (unclamped) of primitive i alone at npix
 * pixels, 0 where it does not contribute (Sec. 3.1), whether or not the
 * pixel's tile is in the primitive's tile set (the tests check with it that
 * the tile set holds every contributing pixel). */
void orc_pair_alpha(void *ctx, int64_t i, int64_t npix, const int32_t *pix, double *ag) {
  orc_ctx *C = (orc_ctx *)ctx;
  const prim_t *p = &C->P[i];
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < npix; ++q) {
    contrib_t c;
    ag[q] = 0.0;
    if (p->valid && eval_pair(C, p, pix[2 * q] + 0.5, pix[2 * q + 1] + 0.5, &c) && c.a_ok && c.z_ok) ag[q] = c.ag;
  }
}

/* For npairs (primitive, pixel) pairs: the conditioning bounds (du, dv) of
 * the primitive's splat-frame coordinates at the pixel (cond_uv), out[2 k],
 * out[2 k + 1]; -1 where the ray misses a surfel's plane.  A gradient
 * through Eq. 1 carries binary32 errors of about that size relative to the
 * footprint; finite-difference checks use pairs where it is small. */
void orc_pair_conditioning(void *ctx, int64_t npairs, const int64_t *ids, const int32_t *pix, double *out) {
  orc_ctx *C = (orc_ctx *)ctx;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < npairs; ++k) {
    const prim_t *p = &C->P[ids[k]];
    const double px = pix[2 * k] + 0.5, py = pix[2 * k + 1] + 0.5;
    double u, v;
    if (p->type == 1) {
      const double dx = px - p->mx, dy = py - p->my;
      u = p->ca * dx + p->cb * dy;
      v = p->cc * dy;
    } else {
      double sol[3];
      if (!surfel_hit(C, p, px, py, sol)) {
        out[2 * k] = out[2 * k + 1] = -1.0;
        continue;
      }
      u = sol[0];
      v = sol[1];
    }
    cond_uv(C, p, px, py, u, v, out + 2 * k, out + 2 * k + 1);
  }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* (4) Adaptive Type Exchange, Sec. 3.2 and App. D, in FP64.                 */
/* mode 0: erank rule with threshold theta (Eq. 3): 3D (t=1) with erank <    */
/*         theta -> 2D; 2D with erank > theta -> 3D.                         */
/* mode 1: flip exactly the primitives whose mask byte is non-zero.          */
/* 3D->2D reparameterises S* = P S P^T, R* = R P^T (Eqs. 4-5); 2D->3D keeps  */
/* every parameter and flips the flag.  Outputs are fresh arrays.            */
/* ------------------------------------------------------------------------ */
double orc_erank(double lsx, double lsy, double lsz) {
  double q[3] = {exp(2 * lsx), exp(2 * lsy), exp(2 * lsz)};
  double s = q[0] + q[1] + q[2];
  double H = 0;
  for (int k = 0; k < 3; ++k) {
    double p = q[k] / s;
    if (p > 0) H -= p * log(p);
  }
  return exp(H);
}

static void qmul(const double a[4], const double b[4], double o[4]) {
  o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

int64_t orc_exchange(int64_t n, const float *log_scales, const float *quats, const uint8_t *types,
                     int mode, double theta, const uint8_t *mask,
                     double *ls_out, double *q_out, uint8_t *t_out) {
  int64_t flips = 0;
  for (int64_t i = 0; i < n; ++i) {
    double ls[3] = {log_scales[3 * i], log_scales[3 * i + 1], log_scales[3 * i + 2]};
    double q[4] = {quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]};
    int t = types[i];
    int flip;
    if (mode == 0) {
      double er = orc_erank(ls[0], ls[1], ls[2]);
      flip = (t == 1) ? (er < theta) : (er > theta);
    } else {
      flip = mask[i] != 0;
    }
    if (flip && t == 1) {
      /* move the least significant scale to z */
      if (ls[2] <= ls[0] && ls[2] <= ls[1]) {
        /* already on z: identity permutation */
      } else if (ls[0] <= ls[1]) {
        /* P_x: S* = diag(sy, sz, sx); R(p) = P_x^T for p = (1/2)(1,1,1,1) */
        double p[4] = {0.5, 0.5, 0.5, 0.5}, o[4];
        double nls[3] = {ls[1], ls[2], ls[0]};
        qmul(q, p, o);
        memcpy(ls, nls, sizeof(nls)); memcpy(q, o, sizeof(o));
      } else {
        /* P_y: S* = diag(sz, sx, sy); R(p) = P_y^T for p = (1/2)(1,-1,-1,-1) */
        double p[4] = {0.5, -0.5, -0.5, -0.5}, o[4];
        double nls[3] = {ls[2], ls[0], ls[1]};
        qmul(q, p, o);
        memcpy(ls, nls, sizeof(nls)); memcpy(q, o, sizeof(o));
      }
    }
    if (flip) { t = 1 - t; flips++; }
    for (int k = 0; k < 3; ++k) ls_out[3 * i + k] = ls[k];
    for (int k = 0; k < 4; ++k) q_out[4 * i + k] = q[k];
    t_out[i] = (uint8_t)t;
  }
  return flips;
}
