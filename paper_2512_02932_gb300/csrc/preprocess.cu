// preprocess.cu -- per-primitive projection of the hybrid rasterizer and its
// backward (EGGS Sec. 3.1, App. C; scale modulation Eqs. 6-7).
//
// Forward, one thread per primitive:
//   binning contract (exact binary32 sequence): camera-space centre, opacity,
//   activated scales, rotation, covered tile rectangle and depth key;
//   render record: projected centre, conic (t=1, Eq. 13) or re-centred
//   inverse homography (t=0, Eqs. 14-15), modulated opacity, SH colour,
//   camera-space normal.
// Backward, one thread per primitive: the record gradient accumulated by
//   render_bwd, chained through the same forward quantities to the raw
//   parameters (means, log-scales, quaternion, opacity logit, SH).
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace hgs {

// ---------------------------------------------------------------------------
// binning contract
// ---------------------------------------------------------------------------
struct Contract {
  float X, Y, Z, iz, xz, yz;
  float alpha, dmax;
  float s[3];
  float qn[4], qinv;  // normalised quaternion, 1/|q|
  float Rq[9];        // rotation of the primitive (row major)
  float a[3][3];      // camera-space axes a[k] = R_cw * column k of Rq
  float s00, s01, s11;                 // t=1: projected covariance
  float e0, e1, f0, f1;                // t=0: re-centred homography block
  uint32_t dbits;
  int tx0, tx1, ty0, ty1;
  float bx0, bx1, by0, by1;  // padded pixel box of the alpha >= alpha_min region
  // tile set (TileSet, common.cuh).  Ellipse mode: the footprint ellipse's
  // centre, chord slope, padded half chord and reciprocal padded half
  // height, heights of its leftmost and rightmost points.  Disc mode (a
  // surfel whose disc reaches the near plane, or whose image conic is
  // degenerate): the disc's centre and axes in pixel-homogeneous camera
  // coordinates.  Rect mode: parameters that overflow binary32.
  float ctrx, ctry, kslope, wp, ihy, yl, yr;
  int mode;  // kSetEllipse, kSetRect or kSetDisc
  float dP[3], dA[3], dB[3];
};

// The contract: a fixed sequence of correctly rounded binary32 operations.
// Returns true if the primitive is binned.
// SETS = false (the backward) skips the tile-set parameters.
template <bool SETS>
__device__ bool run_contract(const float mu[3], const float ls[3], const float q[4], float logit,
                             int type, const CamK &c, const CfgK &f, Contract &o) {
  const float *Rc = c.R;
  o.X = cadd(cadd(cadd(cmul(Rc[0], mu[0]), cmul(Rc[1], mu[1])), cmul(Rc[2], mu[2])), c.t[0]);
  o.Y = cadd(cadd(cadd(cmul(Rc[3], mu[0]), cmul(Rc[4], mu[1])), cmul(Rc[5], mu[2])), c.t[1]);
  o.Z = cadd(cadd(cadd(cmul(Rc[6], mu[0]), cmul(Rc[7], mu[1])), cmul(Rc[8], mu[2])), c.t[2]);
  o.dbits = __float_as_uint(o.Z);
  if (!(o.Z > f.near_z)) return false;
  o.alpha = cdiv(1.0f, cadd(1.0f, contract_exp(-logit)));
  if (!(o.alpha >= f.alpha_min)) return false;
  o.dmax = cmul(2.0f, contract_log(cdiv(o.alpha, f.alpha_min)));
  o.s[0] = contract_exp(ls[0]);
  o.s[1] = contract_exp(ls[1]);
  o.s[2] = contract_exp(ls[2]);
  const float qq = cadd(cadd(cadd(cmul(q[0], q[0]), cmul(q[1], q[1])), cmul(q[2], q[2])),
                        cmul(q[3], q[3]));
  if (!(qq > 0.0f)) return false;
  o.qinv = cdiv(1.0f, csqrt(qq));
  const float w = cmul(q[0], o.qinv), x = cmul(q[1], o.qinv), y = cmul(q[2], o.qinv),
              z = cmul(q[3], o.qinv);
  o.qn[0] = w; o.qn[1] = x; o.qn[2] = y; o.qn[3] = z;
  float *Rq = o.Rq;
  Rq[0] = csub(1.0f, cmul(2.0f, cadd(cmul(y, y), cmul(z, z))));
  Rq[1] = cmul(2.0f, csub(cmul(x, y), cmul(w, z)));
  Rq[2] = cmul(2.0f, cadd(cmul(x, z), cmul(w, y)));
  Rq[3] = cmul(2.0f, cadd(cmul(x, y), cmul(w, z)));
  Rq[4] = csub(1.0f, cmul(2.0f, cadd(cmul(x, x), cmul(z, z))));
  Rq[5] = cmul(2.0f, csub(cmul(y, z), cmul(w, x)));
  Rq[6] = cmul(2.0f, csub(cmul(x, z), cmul(w, y)));
  Rq[7] = cmul(2.0f, cadd(cmul(y, z), cmul(w, x)));
  Rq[8] = csub(1.0f, cmul(2.0f, cadd(cmul(x, x), cmul(y, y))));
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      o.a[k][i] = cadd(cadd(cmul(Rc[3 * i + 0], Rq[0 * 3 + k]), cmul(Rc[3 * i + 1], Rq[1 * 3 + k])),
                       cmul(Rc[3 * i + 2], Rq[2 * 3 + k]));
  o.iz = cdiv(1.0f, o.Z);
  o.xz = cmul(o.X, o.iz);
  o.yz = cmul(o.Y, o.iz);
  const float fx = c.fx, fy = c.fy, cx = c.cx, cy = c.cy;
  float ctrx = 0.f, ctry = 0.f, hx = 0.f, hy = 0.f;
  // tile set: the ellipse's horizontal chord at height y is centred on
  // ctrx + kslope (y - ctry) with half length wch sqrt(1 - ((y - ctry)/hy)^2);
  // its leftmost (rightmost) point lies at y = ctry - yoff (+ yoff)
  float kslope = 0.f, wch = 0.f, yoff = 0.f;
  bool whole = false, full = false, disc = false;
  if (type == 1) {
    const float c0 = cmul(o.s[0], o.s[0]), c1 = cmul(o.s[1], o.s[1]), c2 = cmul(o.s[2], o.s[2]);
    float V[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        V[i][j] = cadd(cadd(cmul(c0, cmul(o.a[0][i], o.a[0][j])), cmul(c1, cmul(o.a[1][i], o.a[1][j]))),
                       cmul(c2, cmul(o.a[2][i], o.a[2][j])));
    const float j00 = cmul(fx, o.iz), j02 = -(cmul(j00, o.xz));
    const float j11 = cmul(fy, o.iz), j12 = -(cmul(j11, o.yz));
    const float t00 = cadd(cmul(j00, V[0][0]), cmul(j02, V[2][0]));
    const float t01 = cadd(cmul(j00, V[0][1]), cmul(j02, V[2][1]));
    const float t02 = cadd(cmul(j00, V[0][2]), cmul(j02, V[2][2]));
    const float t11 = cadd(cmul(j11, V[1][1]), cmul(j12, V[2][1]));
    const float t12 = cadd(cmul(j11, V[1][2]), cmul(j12, V[2][2]));
    o.s00 = cadd(cadd(cmul(j00, t00), cmul(j02, t02)), f.dilation);
    o.s11 = cadd(cadd(cmul(j11, t11), cmul(j12, t12)), f.dilation);
    o.s01 = cadd(cmul(j11, t01), cmul(j12, t02));
    const float det = csub(cmul(o.s00, o.s11), cmul(o.s01, o.s01));
    if (!(det > 0.0f)) return false;
    ctrx = cadd(cmul(fx, o.xz), cx);
    ctry = cadd(cmul(fy, o.yz), cy);
    hx = csqrt(cmul(o.dmax, o.s00));
    hy = csqrt(cmul(o.dmax, o.s11));
    if constexpr (SETS) {
      // det(Sigma') by Cauchy-Binet over the columns t_k = s_k J a_k (a sum of
      // squares: no cancellation for a needle); wch^2 = dmax det / s11
      float tX[3], tY[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        tX[k] = cmul(o.s[k], cadd(cmul(j00, o.a[k][0]), cmul(j02, o.a[k][2])));
        tY[k] = cmul(o.s[k], cadd(cmul(j11, o.a[k][1]), cmul(j12, o.a[k][2])));
      }
      const float m01 = csub(cmul(tX[0], tY[1]), cmul(tY[0], tX[1]));
      const float m02 = csub(cmul(tX[0], tY[2]), cmul(tY[0], tX[2]));
      const float m12 = csub(cmul(tX[1], tY[2]), cmul(tY[1], tX[2]));
      const float x2 = cadd(cadd(cmul(tX[0], tX[0]), cmul(tX[1], tX[1])), cmul(tX[2], tX[2]));
      const float y2 = cadd(cadd(cmul(tY[0], tY[0]), cmul(tY[1], tY[1])), cmul(tY[2], tY[2]));
      const float dil = f.dilation;
      const float detS = cadd(cadd(cadd(cmul(m01, m01), cmul(m02, m02)), cmul(m12, m12)),
                              cadd(cmul(dil, cadd(x2, y2)), cmul(dil, dil)));
      kslope = cdiv(o.s01, o.s11);
      wch = csqrt(cdiv(cmul(o.dmax, detS), o.s11));
      yoff = cdiv(cmul(o.dmax, o.s01), hx);
    }
  } else {
    const float m0x = cmul(o.s[0], o.a[0][0]), m0y = cmul(o.s[0], o.a[0][1]), m0z = cmul(o.s[0], o.a[0][2]);
    const float m1x = cmul(o.s[1], o.a[1][0]), m1y = cmul(o.s[1], o.a[1][1]), m1z = cmul(o.s[1], o.a[1][2]);
    o.e0 = csub(m0x, cmul(o.xz, m0z));
    o.e1 = csub(m1x, cmul(o.xz, m1z));
    o.f0 = csub(m0y, cmul(o.yz, m0z));
    o.f1 = csub(m1y, cmul(o.yz, m1z));
    const float g2 = cadd(cmul(m0z, m0z), cmul(m1z, m1z));
    const float zmin = csub(o.Z, csqrt(cmul(o.dmax, g2)));
    if (!(zmin > f.near_z)) {
      whole = true;
    } else {
      const float e2 = csub(o.X, cmul(o.xz, o.Z));
      const float f2 = csub(o.Y, cmul(o.yz, o.Z));
      const float D22 = csub(cmul(o.dmax, g2), cmul(o.Z, o.Z));
      if (!(D22 < 0.0f)) {
        whole = true;
      } else {
        const float D00 = csub(cmul(o.dmax, cadd(cmul(o.e0, o.e0), cmul(o.e1, o.e1))), cmul(e2, e2));
        const float D02 = csub(cmul(o.dmax, cadd(cmul(o.e0, m0z), cmul(o.e1, m1z))), cmul(e2, o.Z));
        const float D11 = csub(cmul(o.dmax, cadd(cmul(o.f0, o.f0), cmul(o.f1, o.f1))), cmul(f2, f2));
        const float D12 = csub(cmul(o.dmax, cadd(cmul(o.f0, m0z), cmul(o.f1, m1z))), cmul(f2, o.Z));
        const float qx = csub(cmul(D02, D02), cmul(D00, D22));
        const float qy = csub(cmul(D12, D12), cmul(D11, D22));
        if (!(qx >= 0.0f) || !(qy >= 0.0f)) {
          whole = true;
        } else {
          const float nD = -D22;
          const float ox = cdiv(D02, D22), oy = cdiv(D12, D22);
          ctrx = cadd(cmul(fx, cadd(o.xz, ox)), cx);
          ctry = cadd(cmul(fy, cadd(o.yz, oy)), cy);
          hx = cmul(fx, cdiv(csqrt(qx), nD));
          hy = cmul(fy, cdiv(csqrt(qy), nD));
          if constexpr (SETS) {
            // the image ellipse's shape from the dual conic D: Sigma_xy =
            // fx fy (D02 D12 - D01 D22) / D22^2 and det Sigma = fx^2 fy^2 dmax^2
            // det(M)^2 / nD^3, M the re-centred splat frame (det D = -dmax^2
            // det(M)^2)
            const float D01 = csub(cmul(o.dmax, cadd(cmul(o.e0, o.f0), cmul(o.e1, o.f1))), cmul(e2, f2));
            kslope = cdiv(cmul(fx, csub(cmul(D02, D12), cmul(D01, D22))), cmul(fy, qy));
            const float detM = cadd(csub(cmul(o.e0, csub(cmul(o.f1, o.Z), cmul(f2, m1z))),
                                         cmul(o.e1, csub(cmul(o.f0, o.Z), cmul(f2, m0z)))),
                                    cmul(e2, csub(cmul(o.f0, m1z), cmul(o.f1, m0z))));
            wch = cdiv(cmul(cmul(fx, o.dmax), fabsf(detM)), csqrt(cmul(nD, qy)));
            yoff = cdiv(cmul(kslope, cmul(hy, hy)), hx);
          }
        }
      }
    }
    if (whole) {
      full = true;
      disc = true;
      if constexpr (SETS) {
        o.dP[0] = cadd(cmul(fx, o.X), cmul(cx, o.Z));
        o.dP[1] = cadd(cmul(fy, o.Y), cmul(cy, o.Z));
        o.dP[2] = o.Z;
        o.dA[0] = cadd(cmul(fx, m0x), cmul(cx, m0z));
        o.dA[1] = cadd(cmul(fy, m0y), cmul(cy, m0z));
        o.dA[2] = m0z;
        o.dB[0] = cadd(cmul(fx, m1x), cmul(cx, m1z));
        o.dB[1] = cadd(cmul(fy, m1y), cmul(cy, m1z));
        o.dB[2] = m1z;
      }
      // The disc reaches the near plane (or its image conic is degenerate):
      // a contributing hit lies inside the disc's camera-space extents R at a
      // depth in (near, Z + R_z], which bounds x/z and y/z.
      const float sd = csqrt(o.dmax);
      const float Rx = cmul(sd, csqrt(cadd(cmul(m0x, m0x), cmul(m1x, m1x))));
      const float Ry = cmul(sd, csqrt(cadd(cmul(m0y, m0y), cmul(m1y, m1y))));
      const float zhi = cadd(o.Z, cmul(sd, csqrt(g2)));
      const float xl = csub(o.X, Rx), xh = cadd(o.X, Rx), yl = csub(o.Y, Ry), yh = cadd(o.Y, Ry);
      const float nxl = xl >= 0.0f ? cdiv(xl, zhi) : cdiv(xl, f.near_z);
      const float nxh = xh >= 0.0f ? cdiv(xh, f.near_z) : cdiv(xh, zhi);
      const float nyl = yl >= 0.0f ? cdiv(yl, zhi) : cdiv(yl, f.near_z);
      const float nyh = yh >= 0.0f ? cdiv(yh, f.near_z) : cdiv(yh, zhi);
      const float ilx = cadd(cmul(fx, nxl), cx), ihx = cadd(cmul(fx, nxh), cx);
      const float ily = cadd(cmul(fy, nyl), cy), ihy = cadd(cmul(fy, nyh), cy);
      ctrx = cmul(0.5f, cadd(ilx, ihx));
      ctry = cmul(0.5f, cadd(ily, ihy));
      hx = cmul(0.5f, csub(ihx, ilx));
      hy = cmul(0.5f, csub(ihy, ily));
      whole = false;
    }
  }
  if (whole) {
    o.tx0 = 0; o.tx1 = (c.W - 1) / kTile;
    o.ty0 = 0; o.ty1 = (c.H - 1) / kTile;
    o.bx0 = o.by0 = -1e30f;
    o.bx1 = o.by1 = 1e30f;
    full = true;
  } else {
    const float px = pad_extent(hx), py = pad_extent(hy);
    o.bx0 = csub(ctrx, px); o.bx1 = cadd(ctrx, px);
    o.by0 = csub(ctry, py); o.by1 = cadd(ctry, py);
    if (!pixel_tiles(o.bx0, o.bx1, c.W, &o.tx0, &o.tx1)) return false;
    if (!pixel_tiles(o.by0, o.by1, c.H, &o.ty0, &o.ty1)) return false;
  }
  if constexpr (!SETS) return true;
  if (disc) {
    bool fin = isfinite(o.dmax);
#pragma unroll
    for (int k = 0; k < 3; ++k) fin = fin && isfinite(o.dP[k]) && isfinite(o.dA[k]) && isfinite(o.dB[k]);
    o.mode = fin ? kSetDisc : kSetRect;
    return true;
  }
  // padded chord parameters: the half chord by pad_extent plus 2^-10 hx for
  // the rounding of kslope (y - ctry), the half height by pad_extent (its
  // reciprocal is stored)
  o.ctrx = ctrx;
  o.ctry = ctry;
  o.kslope = kslope;
  o.wp = cadd(pad_extent(wch), cmul(hx, 0x1p-10f));
  const float hyp = pad_extent(hy);
  o.ihy = cdiv(1.0f, hyp);
  o.yl = csub(ctry, yoff);
  o.yr = cadd(ctry, yoff);
  const bool bad = !(isfinite(o.kslope) && isfinite(o.wp) && isfinite(o.yl) && isfinite(o.yr) && hyp > 0.0f &&
                     isfinite(o.ihy));
  o.mode = (full || bad) ? kSetRect : kSetEllipse;
  return true;
}

// ---------------------------------------------------------------------------
// real spherical harmonics (degree <= 3), as homogeneous polynomials in the
// unit view direction (x, y, z); constants are the real-SH normalisations
// (Condon-Shortley phase kept), e.g. k1 = sqrt(3/(4 pi)).
// ---------------------------------------------------------------------------
#define SH_K0 0.28209479177387814f   /* 1/(2 sqrt(pi)) */
#define SH_K1 0.48860251190291992f   /* sqrt(3/(4 pi)) */
#define SH_K2A 1.0925484305920792f   /* sqrt(15/pi)/2 */
#define SH_K2B 0.31539156525252005f  /* sqrt(5/pi)/4 */
#define SH_K2C 0.54627421529603959f  /* sqrt(15/pi)/4 */
#define SH_K3A 0.59004358992664352f  /* sqrt(35/(2 pi))/4 */
#define SH_K3B 2.8906114426405538f   /* sqrt(105/pi)/2 */
#define SH_K3C 0.45704579946446572f  /* sqrt(21/(2 pi))/4 */
#define SH_K3D 0.37317633259011540f  /* sqrt(7/pi)/4 */
#define SH_K3E 1.4453057213202769f   /* sqrt(105/pi)/4 */

template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float *Y) {
  Y[0] = SH_K0;
  if (DEG >= 1) {
    Y[1] = -SH_K1 * y;
    Y[2] = SH_K1 * z;
    Y[3] = -SH_K1 * x;
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SH_K2A * x * y;
    Y[5] = -SH_K2A * y * z;
    Y[6] = SH_K2B * (2.f * zz - xx - yy);
    Y[7] = -SH_K2A * x * z;
    Y[8] = SH_K2C * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -SH_K3A * y * (3.f * xx - yy);
      Y[10] = SH_K3B * x * y * z;
      Y[11] = -SH_K3C * y * (4.f * zz - xx - yy);
      Y[12] = SH_K3D * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -SH_K3C * x * (4.f * zz - xx - yy);
      Y[14] = SH_K3E * z * (xx - yy);
      Y[15] = -SH_K3A * x * (xx - 3.f * yy);
    }
  }
}

// d/d(x,y,z) of sum_k w_k Y_k
template <int DEG>
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float *w, float g[3]) {
  g[0] = g[1] = g[2] = 0.f;
  if (DEG >= 1) {
    g[1] += -SH_K1 * w[1];
    g[2] += SH_K1 * w[2];
    g[0] += -SH_K1 * w[3];
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    g[0] += SH_K2A * y * w[4];
    g[1] += SH_K2A * x * w[4];
    g[1] += -SH_K2A * z * w[5];
    g[2] += -SH_K2A * y * w[5];
    g[0] += -2.f * SH_K2B * x * w[6];
    g[1] += -2.f * SH_K2B * y * w[6];
    g[2] += 4.f * SH_K2B * z * w[6];
    g[0] += -SH_K2A * z * w[7];
    g[2] += -SH_K2A * x * w[7];
    g[0] += 2.f * SH_K2C * x * w[8];
    g[1] += -2.f * SH_K2C * y * w[8];
    if (DEG >= 3) {
      g[0] += -6.f * SH_K3A * x * y * w[9];
      g[1] += -SH_K3A * (3.f * xx - 3.f * yy) * w[9];
      g[0] += SH_K3B * y * z * w[10];
      g[1] += SH_K3B * x * z * w[10];
      g[2] += SH_K3B * x * y * w[10];
      g[0] += 2.f * SH_K3C * x * y * w[11];
      g[1] += -SH_K3C * (4.f * zz - xx - 3.f * yy) * w[11];
      g[2] += -8.f * SH_K3C * y * z * w[11];
      g[0] += -6.f * SH_K3D * x * z * w[12];
      g[1] += -6.f * SH_K3D * y * z * w[12];
      g[2] += SH_K3D * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
      g[0] += -SH_K3C * (4.f * zz - 3.f * xx - yy) * w[13];
      g[1] += 2.f * SH_K3C * x * y * w[13];
      g[2] += -8.f * SH_K3C * x * z * w[13];
      g[0] += 2.f * SH_K3E * x * z * w[14];
      g[1] += -2.f * SH_K3E * y * z * w[14];
      g[2] += SH_K3E * (xx - yy) * w[14];
      g[0] += -SH_K3A * (3.f * xx - 3.f * yy) * w[15];
      g[1] += 6.f * SH_K3A * x * y * w[15];
    }
  }
}

template <int DEG>
__device__ __forceinline__ void load_sh(const float *sh, int64_t i, float *f) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
  const float *p = sh + (int64_t)i * NB * 3;
  if constexpr (DEG == 0) {
    f[0] = __ldg(p); f[1] = __ldg(p + 1); f[2] = __ldg(p + 2);
  } else {
    // (DEG+1)^2 * 3 floats = 12, 27 or 48; rows are 16-byte aligned only for
    // degrees 1 and 3 (48 and 192 bytes); degree 2 (108 bytes) loads scalars
    if constexpr ((NB * 3) % 4 == 0) {
      const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
      for (int k = 0; k < NB * 3 / 4; ++k) {
        const float4 v = __ldg(p4 + k);
        f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < NB * 3; ++k) f[k] = __ldg(p + k);
    }
  }
}

// Visit the SH row p coefficient by coefficient (fn(k, f_k0, f_k1, f_k2)),
// loading a few 16-byte pieces at a time so the row is never held whole.
template <int DEG, class Fn>
__device__ __forceinline__ void sh_visit(const float *p, Fn &&fn) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
  if constexpr ((NB * 3) % 4 == 0) {
    // four coefficients (12 floats, three float4) per step
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int c = 0; c < NB / 4; ++c) {
      const float4 a = __ldg(p4 + 3 * c), b = __ldg(p4 + 3 * c + 1), d = __ldg(p4 + 3 * c + 2);
      fn(4 * c + 0, a.x, a.y, a.z);
      fn(4 * c + 1, a.w, b.x, b.y);
      fn(4 * c + 2, b.z, b.w, d.x);
      fn(4 * c + 3, d.y, d.z, d.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NB; ++k) fn(k, __ldg(p + 3 * k), __ldg(p + 3 * k + 1), __ldg(p + 3 * k + 2));
  }
}

// a d - b c with one rounding error (Kahan's FMA algorithm)
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
  const float w = __fmul_rn(b, c);
  const float e = __fmaf_rn(-b, c, w);
  return __fadd_rn(__fmaf_rn(a, d, -w), e);
}

// Projected covariance of a 3D Gaussian from its factor T = J W R S (2x3):
// Sigma' = T T^T + dilation I, with det(T T^T) by the Cauchy-Binet sum of the
// squared 2x2 minors (a sum of squares: no cancellation, so the conic of a
// needle-like footprint stays accurate in binary32).
struct Cov2 {
  float s00, s01, s11, det;
};

__device__ __forceinline__ Cov2 projected_cov(const Contract &o, const CamK &c, float dil) {
  const float iz = o.iz;
  const float j00 = c.fx * iz, j02 = -c.fx * o.X * iz * iz;
  const float j11 = c.fy * iz, j12 = -c.fy * o.Y * iz * iz;
  float tx[3], ty[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    tx[k] = o.s[k] * fmaf(j00, o.a[k][0], j02 * o.a[k][2]);
    ty[k] = o.s[k] * fmaf(j11, o.a[k][1], j12 * o.a[k][2]);
  }
  Cov2 v;
  const float x2 = tx[0] * tx[0] + tx[1] * tx[1] + tx[2] * tx[2];
  const float y2 = ty[0] * ty[0] + ty[1] * ty[1] + ty[2] * ty[2];
  v.s01 = tx[0] * ty[0] + tx[1] * ty[1] + tx[2] * ty[2];
  const float m01 = tx[0] * ty[1] - ty[0] * tx[1];
  const float m02 = tx[0] * ty[2] - ty[0] * tx[2];
  const float m12 = tx[1] * ty[2] - ty[1] * tx[2];
  v.s00 = x2 + dil;
  v.s11 = y2 + dil;
  v.det = (m01 * m01 + m02 * m02 + m12 * m12) + dil * (x2 + y2) + dil * dil;
  return v;
}

// write one primitive's SH row (zeros if v is null); 16-byte stores where the
// row is 16-byte aligned (degrees 1 and 3)
template <int DEG>
__device__ __forceinline__ void store_sh(float *dst, const float *v) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
  if constexpr ((NB * 3) % 4 == 0) {
    float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int k = 0; k < NB * 3 / 4; ++k)
      d4[k] = v ? make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3])
                : make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
#pragma unroll
    for (int k = 0; k < NB * 3; ++k) dst[k] = v ? v[k] : 0.0f;
  }
}

__device__ __forceinline__ int normal_axis(int type, const float ls[3]) {
  if (type == 0) return 2;
  if (ls[2] <= ls[0] && ls[2] <= ls[1]) return 2;
  return ls[0] <= ls[1] ? 0 : 1;
}

// camera-space axis k of the primitive, selected without dynamic indexing
__device__ __forceinline__ void axis_of(const Contract &o, int k, float &x, float &y, float &z) {
  x = k == 0 ? o.a[0][0] : (k == 1 ? o.a[1][0] : o.a[2][0]);
  y = k == 0 ? o.a[0][1] : (k == 1 ? o.a[1][1] : o.a[2][1]);
  z = k == 0 ? o.a[0][2] : (k == 1 ? o.a[1][2] : o.a[2][2]);
}

__device__ __forceinline__ void load_params(const PrepArgs &a, int64_t i, float mu[3], float ls[3],
                                            float q[4], float &logit, int &type) {
  mu[0] = __ldg(a.means + 3 * i); mu[1] = __ldg(a.means + 3 * i + 1); mu[2] = __ldg(a.means + 3 * i + 2);
  ls[0] = __ldg(a.log_scales + 3 * i); ls[1] = __ldg(a.log_scales + 3 * i + 1);
  ls[2] = __ldg(a.log_scales + 3 * i + 2);
  const float4 qv = __ldg(reinterpret_cast<const float4 *>(a.quats) + i);
  q[0] = qv.x; q[1] = qv.y; q[2] = qv.z; q[3] = qv.w;
  logit = __ldg(a.logits + i);
  type = __ldg(a.types + i) ? 1 : 0;
}

// 2D opacity modulation (Eqs. 6-7): alpha* = alpha exp(-lambda s_z*),
// s_z* = sigmoid((s_z - theta_z)/T_z) s_z.  Returns alpha*, and the factors
// the backward needs.
__device__ __forceinline__ float modulate(float alpha, float sz, const CfgK &f, float *gate,
                                          float *fac) {
  const float g = 1.0f / (1.0f + expf(-(sz - f.theta_z) / f.T_z));
  const float e = expf(-f.lambda_z * (g * sz));
  *gate = g;
  *fac = e;
  return alpha * e;
}

// Projected centre fx X/Z + cx, fy Y/Z + cy as double-floats (hi + lo), from
// the binary32 inputs with error-free products and sums (~44 bits).
__device__ __forceinline__ void df_dot(const float r[3], const float mu[3], float t, float &hi, float &lo) {
  float h = t, l = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float p, pe, s, se;
    two_prod(r[k], mu[k], p, pe);
    two_sum(h, p, s, se);
    h = s;
    l = __fadd_rn(l, __fadd_rn(pe, se));
  }
  two_sum(h, l, hi, lo);
}

__device__ __forceinline__ void df_centre(const CamK &c, const float mu[3], float &xh, float &xl,
                                          float &yh, float &yl) {
  float Xh, Xl, Yh, Yl, Zh, Zl;
  df_dot(c.R + 0, mu, c.t[0], Xh, Xl);
  df_dot(c.R + 3, mu, c.t[1], Yh, Yl);
  df_dot(c.R + 6, mu, c.t[2], Zh, Zl);
  // x/z: q1 + q2 with q2 = (X - q1 Z) / Z
  auto ddiv = [&](float nh, float nl, float &qh, float &ql) {
    const float q1 = __fdiv_rn(nh, Zh);
    float p, pe;
    two_prod(q1, Zh, p, pe);
    const float r = __fsub_rn(__fsub_rn(__fsub_rn(nh, p), pe), __fmul_rn(q1, Zl));
    const float q2 = __fdiv_rn(__fadd_rn(r, nl), Zh);
    two_sum(q1, q2, qh, ql);
  };
  auto dscale = [&](float f, float off, float qh, float ql, float &oh, float &ol) {
    float p, pe, s, se;
    two_prod(f, qh, p, pe);
    two_sum(p, off, s, se);
    two_sum(s, __fadd_rn(__fadd_rn(se, pe), __fmul_rn(f, ql)), oh, ol);
  };
  float qxh, qxl, qyh, qyl;
  ddiv(Xh, Xl, qxh, qxl);
  ddiv(Yh, Yl, qyh, qyl);
  dscale(c.fx, c.cx, qxh, qxl, xh, xl);
  dscale(c.fy, c.cy, qyh, qyl, yh, yl);
}

// two halves rounded outwards (lo down, hi up), packed in a float's bits
__device__ __forceinline__ float pack_box(float lo, float hi) {
  lo = fmaxf(lo, -65504.0f);
  hi = fminf(hi, 65504.0f);
  const __half a = __float2half_rd(lo), b = __float2half_ru(hi);
  const uint32_t u = (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
  return __uint_as_float(u);
}

// ---------------------------------------------------------------------------
// forward kernel
// ---------------------------------------------------------------------------
// Ask L2 for a primitive's SH row ahead of its use, so that the row's DRAM
// latency overlaps the contract arithmetic: only for primitives that pass a
// cheap guess at the contract's culls (in front of the near plane, opacity
// above alpha_min, centre within a margin of the image).  A hint only.
template <int DEG>
__device__ __forceinline__ void prefetch_sh(const PrepArgs &a, int64_t i, const float (&mu)[3], float logit) {
  if constexpr (DEG > 0) {
    constexpr int NB = (DEG + 1) * (DEG + 1);
    const CamK &c = a.cam;
    const float X = fmaf(c.R[0], mu[0], fmaf(c.R[1], mu[1], fmaf(c.R[2], mu[2], c.t[0])));
    const float Y = fmaf(c.R[3], mu[0], fmaf(c.R[4], mu[1], fmaf(c.R[5], mu[2], c.t[1])));
    const float Z = fmaf(c.R[6], mu[0], fmaf(c.R[7], mu[1], fmaf(c.R[8], mu[2], c.t[2])));
    const bool front = Z > a.cfg.near_z && logit > -5.6f;
    const float W = (float)c.W, H = (float)c.H;
    const bool near_view = fabsf(fmaf(c.fx, X, (c.cx - 0.5f * W) * Z)) < W * Z &&
                           fabsf(fmaf(c.fy, Y, (c.cy - 0.5f * H) * Z)) < H * Z;
    if (front && near_view) {
      const char *p = reinterpret_cast<const char *>(a.sh + (int64_t)i * NB * 3);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
      if (NB * 12 > 96) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + 96));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p + NB * 12 - 4));
    }
  }
}

// One primitive's parameters as loaded.
struct PrimIn {
  float mu[3], ls[3], q[4], logit;
  int type;
};

// Contract part of the forward for primitive i: the depth key, and, if the
// rectangle is not empty, the tile-set parameters (ts) and the number of
// tile rows of the rectangle (0 if not binned).
__device__ __forceinline__ int contract_part(const PrepArgs &a, int64_t i, int row_off, const PrimIn &p,
                                             Contract &o, TileSet &ts) {
  const bool binned = run_contract<true>(p.mu, p.ls, p.q, p.logit, p.type, a.cam, a.cfg, o);
  a.depth_key[i] = o.dbits;
  if (!binned) return 0;
  const float fl = __uint_as_float(tileset_flags(o.mode, row_off, a.cam.W));
  if (o.mode == kSetDisc) {
    ts.t0 = make_float4(o.dP[0], o.dP[1], o.dP[2], o.dmax);
    ts.t1 = make_float4(o.dA[0], o.dA[1], o.dA[2], a.cfg.near_z);
    ts.t2 = make_float4(o.dB[0], o.dB[1], o.dB[2], fl);
  } else {
    ts.t0 = make_float4(o.ctrx, o.ctry, o.kslope, o.wp);
    ts.t1 = make_float4(o.ihy, o.yl, o.yr, 0.0f);
    ts.t2 = make_float4(0.0f, 0.0f, 0.0f, fl);
  }
  // written now (only read for a primitive whose set is not empty)
  float4 *tsd = reinterpret_cast<float4 *>(a.tileset) + 3 * i;
  tsd[0] = ts.t0;
  tsd[1] = ts.t1;
  tsd[2] = ts.t2;
  return o.ty1 - o.ty0 + 1;
}

// The size of each lane's tile set, counted by the warp's lanes together:
// the (primitive, tile row) pairs of the warp are spread over the lanes (a
// lane finds the primitive of its pair by a binary search over the exclusive
// prefix of the lanes' row counts), so a primitive spanning many rows does
// not hold up the other lanes.  Every lane of the warp calls it; sts and scnt
// are the warp's shared-memory slots.
__device__ __forceinline__ uint32_t warp_set_count(const TileSet &ts, int tx0, int tx1, int ty0, int nrows,
                                                   TileSet *sts, uint32_t *scnt) {
  const int lane = threadIdx.x & 31;
  sts[lane] = ts;
  scnt[lane] = 0u;
  uint32_t incl = (uint32_t)nrows;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const uint32_t rel = incl - (uint32_t)nrows;
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  for (uint32_t kb = 0; kb < total; kb += 32) {  // warp-uniform trip count
    const uint32_t k = kb + lane;
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint32_t pr = __shfl_sync(0xffffffffu, rel, lo + step);
      if (pr <= k) lo += step;
    }
    const uint32_t orel = __shfl_sync(0xffffffffu, rel, lo);
    const int otx0 = __shfl_sync(0xffffffffu, tx0, lo), otx1 = __shfl_sync(0xffffffffu, tx1, lo);
    const int oty0 = __shfl_sync(0xffffffffu, ty0, lo);
    if (k < total) {
      int c0, c1;
      if (row_span(sts[lo], oty0 + (int)(k - orel), otx0, otx1, &c0, &c1))
        atomicAdd(&scnt[lo], (uint32_t)(c1 - c0 + 1));
    }
  }
  __syncwarp();
  return scnt[lane];
}

// The rest of the forward for a primitive whose contract ran: its binning
// outputs (a primitive whose tile set is empty is not binned) and its render
// record.
template <int DEG>
__device__ __forceinline__ void finish_one(const PrepArgs &a, int64_t i, int row_off, const PrimIn &p,
                                           const Contract &o, uint32_t count) {
  if (count == 0u) {
    a.touched[i] = 0u;
    reinterpret_cast<uint2 *>(a.rect)[i] = make_uint2(0u, 0u);
    return;
  }
  const float(&mu)[3] = p.mu;
  const float(&ls)[3] = p.ls;
  const int type = p.type;
  a.touched[i] = count;
  reinterpret_cast<uint2 *>(a.rect)[i] =
      make_uint2((uint32_t)o.tx0 | ((uint32_t)o.tx1 << 16),
                 (uint32_t)(o.ty0 + row_off) | ((uint32_t)(o.ty1 + row_off) << 16));

  const CamK &c = a.cam;
  // colour (Sec. 3.1): SH decoded along the view direction
  constexpr int NB = (DEG + 1) * (DEG + 1);
  float dx = mu[0] - c.campos[0], dy = mu[1] - c.campos[1], dz = mu[2] - c.campos[2];
  const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
  dx *= il; dy *= il; dz *= il;
  float Y[NB];
  sh_eval<DEG>(dx, dy, dz, Y);
  float col[3] = {0.5f, 0.5f, 0.5f};
  sh_visit<DEG>(a.sh + i * NB * 3, [&](int k, float f0, float f1, float f2) {
    col[0] = fmaf(f0, Y[k], col[0]);
    col[1] = fmaf(f1, Y[k], col[1]);
    col[2] = fmaf(f2, Y[k], col[2]);
  });
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) col[ch] = fmaxf(col[ch], 0.0f);
  // normal: smallest-scale axis (z for a surfel), facing the camera
  const int kn = normal_axis(type, ls);
  float n0, n1, n2;
  axis_of(o, kn, n0, n1, n2);
  if (n0 * o.X + n1 * o.Y + n2 * o.Z > 0.0f) { n0 = -n0; n1 = -n1; n2 = -n2; }
  float ctrx, ctrx_lo, ctry, ctry_lo;
  df_centre(c, mu, ctrx, ctrx_lo, ctry, ctry_lo);
  Rec r;
  if (type == 1) {
    // Eq. 1 as d = |W (dx, dy)|^2 with W the Cholesky factor of the conic:
    // W = [[sqrt(s11/det), -s01/sqrt(s11 det)], [0, 1/sqrt(s11)]]
    const Cov2 cv = projected_cov(o, c, a.cfg.dilation);
    const float w00 = sqrtf(cv.s11 / cv.det);
    const float w01 = -cv.s01 * rsqrtf(cv.s11 * cv.det);
    const float w11 = rsqrtf(cv.s11);
    const bool ok = cv.det > 0.0f && cv.s11 > 0.0f && isfinite(w00) && isfinite(w01) && isfinite(w11);
    r.r0 = make_float4(ctrx, ctry, o.Z, ok ? o.alpha : 0.0f);
    r.r1 = ok ? make_float4(w00, w01, w11, 0.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
    r.r2 = make_float4(0.0f, 0.0f, col[0], col[1]);
  } else {
    float gate, fac;
    const float am = modulate(o.alpha, o.s[2], a.cfg, &gate, &fac);
    const float m0z = o.s[0] * o.a[0][2], m1z = o.s[1] * o.a[1][2];
    const float detE = det2(o.e0, o.e1, o.f0, o.f1);
    const float ie = 1.0f / detE;
    const float E00 = o.f1 * ie, E01 = -o.e1 * ie, E10 = -o.f0 * ie, E11 = o.e0 * ie;
    const float ifx = 1.0f / c.fx, ify = 1.0f / c.fy;
    float Q00 = o.Z * E00 * ifx, Q01 = o.Z * E01 * ify, Q10 = o.Z * E10 * ifx, Q11 = o.Z * E11 * ify;
    float Q20 = -(m0z * E00 + m1z * E10) * ifx, Q21 = -(m0z * E01 + m1z * E11) * ify;
    float as = -am;
    const bool finite = isfinite(Q00) && isfinite(Q01) && isfinite(Q10) && isfinite(Q11) &&
                        isfinite(Q20) && isfinite(Q21);
    if (!finite) {
      // edge-on surfel (plane through the camera centre): it covers no pixel;
      // a zero-opacity record keeps the binned list intact
      Q00 = Q01 = Q10 = Q11 = Q20 = Q21 = 0.0f;
      as = -0.0f;
    }
    r.r0 = make_float4(ctrx, ctry, o.Z, as);
    r.r1 = make_float4(Q00, Q01, Q10, Q11);
    r.r2 = make_float4(Q20, Q21, col[0], col[1]);
  }
  r.r3 = make_float4(col[2], n0, n1, n2);
  r.r4 = make_float4(ctrx_lo, ctry_lo, pack_box(o.bx0, o.bx1), pack_box(o.by0, o.by1));
  float4 *dst = reinterpret_cast<float4 *>(a.rec) + kRecF4 * i;
  dst[0] = r.r0; dst[1] = r.r1; dst[2] = r.r2; dst[3] = r.r3; dst[4] = r.r4;
}

template <int DEG>
__global__ void __launch_bounds__(256, 3) preprocess_fwd_kernel(PrepArgs a) {
  __shared__ TileSet sts[8][32];
  __shared__ uint32_t scnt[8][32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = i < a.n;
  if (__all_sync(0xffffffffu, !in)) return;
  const int warp = threadIdx.x >> 5;
  PrimIn p;
  Contract o;
  TileSet ts;
  int nrows = 0;
  if (in) {
    load_params(a, i, p.mu, p.ls, p.q, p.logit, p.type);
    prefetch_sh<DEG>(a, i, p.mu, p.logit);
    nrows = contract_part(a, i, 0, p, o, ts);
  }
  const uint32_t count = warp_set_count(ts, o.tx0, o.tx1, o.ty0, nrows, sts[warp], scnt[warp]);
  if (in) finish_one<DEG>(a, i, 0, p, o, count);
}

// Batched: the requests' primitives are concatenated; request r covers global
// rows [base[r], base[r+1]) and its outputs start at row base[r]; the tile
// rectangle's rows are shifted by row_off[r] (the batched render stacks the
// requests' tile grids vertically).
__global__ void __launch_bounds__(256) preprocess_batch_kernel(BatchPrepArgs b) {
  __shared__ TileSet sts[8][32];
  __shared__ uint32_t scnt[8][32];
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = g < b.base[b.nreq];
  if (__all_sync(0xffffffffu, !in)) return;
  const int warp = threadIdx.x >> 5;
  int r = 0;
  if (in)
    while (r + 1 < b.nreq && g >= b.base[r + 1]) ++r;
  const int64_t i = g - b.base[r];
  const PrepArgs &a = b.req[r];
  PrimIn p;
  Contract o;
  TileSet ts;
  int nrows = 0;
  if (in) {
    load_params(a, i, p.mu, p.ls, p.q, p.logit, p.type);
    nrows = contract_part(a, i, b.row_off[r], p, o, ts);
  }
  const uint32_t count = warp_set_count(ts, o.tx0, o.tx1, o.ty0 + b.row_off[r], nrows, sts[warp], scnt[warp]);
  if (!in) return;
  switch (b.deg[r]) {
    case 0: finish_one<0>(a, i, b.row_off[r], p, o, count); break;
    case 1: finish_one<1>(a, i, b.row_off[r], p, o, count); break;
    case 2: finish_one<2>(a, i, b.row_off[r], p, o, count); break;
    default: finish_one<3>(a, i, b.row_off[r], p, o, count); break;
  }
}

// ---------------------------------------------------------------------------
// backward kernel
// ---------------------------------------------------------------------------
// Raw-parameter gradient of one primitive.  The SH part is dv (x) Y: the
// colour gradient per channel, zero where the colour was clamped, times the
// basis at the view direction.
struct PGrad {
  float mu[3], ls[3], logit, dv[3];
  float4 q;
};

// What the backward needs of one primitive besides its record gradient.
// STREAM: the SH row is read again where it is needed (twice), never held
// whole, which keeps the one-set backward at 80 registers; else (the
// three-set backward, which runs the chain three times) it is held.
template <int DEG, bool STREAM>
struct BwdCtx {
  static constexpr int NB = (DEG + 1) * (DEG + 1);
  float mu[3], ls[3];
  int type;
  Contract o;
  const float *f;                    // the primitive's SH row
  float fr[STREAM ? 1 : NB * 3];     // its copy in registers (not STREAM)
  float Yb[NB];
  float ux, uy, uz, il;
  bool cpos[3];  // colour channel not clamped at 0
  template <class Fn>
  __device__ __forceinline__ void visit_sh(Fn &&fn) const {
    if constexpr (STREAM) {
      sh_visit<DEG>(f, fn);
    } else {
#pragma unroll
      for (int k = 0; k < NB; ++k) fn(k, fr[3 * k], fr[3 * k + 1], fr[3 * k + 2]);
    }
  }
};


template <int DEG, bool STREAM>
__device__ __forceinline__ void bwd_ctx(const PrepArgs &a, int64_t i, BwdCtx<DEG, STREAM> &x) {
  constexpr int NB = BwdCtx<DEG, STREAM>::NB;
  float q[4], logit;
  load_params(a, i, x.mu, x.ls, q, logit, x.type);
  run_contract<false>(x.mu, x.ls, q, logit, x.type, a.cam, a.cfg, x.o);
  x.f = a.sh + i * NB * 3;
  if constexpr (!STREAM) load_sh<DEG>(a.sh, i, x.fr);
  const CamK &c = a.cam;
  const float vx = x.mu[0] - c.campos[0], vy = x.mu[1] - c.campos[1], vz = x.mu[2] - c.campos[2];
  x.il = rsqrtf(vx * vx + vy * vy + vz * vz);
  x.ux = vx * x.il; x.uy = vy * x.il; x.uz = vz * x.il;
  sh_eval<DEG>(x.ux, x.uy, x.uz, x.Yb);
  float v[3] = {0.5f, 0.5f, 0.5f};
  x.visit_sh([&](int k, float f0, float f1, float f2) {
    v[0] = fmaf(f0, x.Yb[k], v[0]);
    v[1] = fmaf(f1, x.Yb[k], v[1]);
    v[2] = fmaf(f2, x.Yb[k], v[2]);
  });
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) x.cpos[ch] = v[ch] > 0.0f;
}

// The chain from a record gradient G (layout: common.cuh) to the raw
// parameters: projection (App. C), camera, rotation, activations and the SH
// colour.  Linear in G.
template <int DEG, bool STREAM>
__device__ __forceinline__ PGrad chain_grad(const PrepArgs &a, const BwdCtx<DEG, STREAM> &ctx,
                                            const float (&G)[kGradW]) {
  constexpr int NB = BwdCtx<DEG, STREAM>::NB;
  const CamK &c = a.cam;
  const Contract &o = ctx.o;
  const int type = ctx.type;
  const float(&ls)[3] = ctx.ls;
  float dX = 0.f, dY = 0.f, dZ = G[6];
  float dA[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  float dls[3] = {0.f, 0.f, 0.f};
  float dalpha = 0.f;
  const float fx = c.fx, fy = c.fy;
  const float X = o.X, Y = o.Y, Z = o.Z, iz = o.iz;

  // normal
  {
    const int kn = normal_axis(type, ls);
    float ax, ay, az;
    axis_of(o, kn, ax, ay, az);
    const float sg = (ax * X + ay * Y + az * Z > 0.0f) ? -1.f : 1.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float w = (k == kn) ? sg : 0.0f;
      dA[k][0] += w * G[13];
      dA[k][1] += w * G[14];
      dA[k][2] += w * G[15];
    }
  }
  const float dxc = G[4], dyc = G[5];
  if (type == 1) {
    dalpha = G[0];
    // Footprint factor T = J A S, column t_k = s_k J a_k (a_k the camera-space
    // axes), Sigma' = T T^T + dilation I, conic C = Sigma'^-1 = W^T W.  The
    // record gradient (slots 7-9) is Hg = dL/dH for the shape H in footprint
    // coordinates (u, v) = W (dx, dy); with w_k = W t_k (so C t_k = W^T w_k)
    // and Q_jk = w_j^T Hg w_k, the derivatives of L through T are
    //   dL/dlog s_k = -2 Q_kk
    //   dL/da_k     = -2 sum_j (s_k / s_j) Q_jk a_j      (a_j orthonormal)
    //   dL/dX = (2/Z) sum_j R_j a_jx / s_j,  dL/dY likewise with a_jy,
    //   dL/dZ = (2/Z) (tr Q + sum_j R_j a_jz / s_j),  R_j = sum_k Q_jk s_k a_kz,
    // using J e_x = (fx/Z) e_x, J e_y = (fy/Z) e_y, J e_z = -Z (dJ/dZ part)
    // and J a_j = t_j / s_j.  No term multiplies the conic's large
    // eigenvalue into a needle's long axis, so binary32 keeps these
    // accurate where dL/dC contracted with T would cancel.
    const Cov2 cv = projected_cov(o, c, a.cfg.dilation);
    const float w00 = sqrtf(cv.s11 / cv.det);
    const float w01 = -cv.s01 * rsqrtf(cv.s11 * cv.det);
    const float w11 = rsqrtf(cv.s11);
    const float h00 = G[7], h01 = 0.5f * G[8], h11 = G[9];
    const float j00 = fx * iz, j02 = -fx * X * iz * iz, j11 = fy * iz, j12 = -fy * Y * iz * iz;
    float wu[3], wv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float tx = o.s[k] * fmaf(j00, o.a[k][0], j02 * o.a[k][2]);
      const float ty = o.s[k] * fmaf(j11, o.a[k][1], j12 * o.a[k][2]);
      wu[k] = fmaf(w00, tx, w01 * ty);
      wv[k] = w11 * ty;
    }
    float Q[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float pu = fmaf(h00, wu[k], h01 * wv[k]), pv = fmaf(h01, wu[k], h11 * wv[k]);
#pragma unroll
      for (int j = 0; j < 3; ++j) Q[j][k] = fmaf(wu[j], pu, wv[j] * pv);
    }
    float is[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) is[k] = 1.0f / o.s[k];
    float rx = 0.f, ry = 0.f, rz = 0.f, tr = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float Rj = Q[j][0] * o.s[0] * o.a[0][2] + Q[j][1] * o.s[1] * o.a[1][2] + Q[j][2] * o.s[2] * o.a[2][2];
      rx = fmaf(Rj * is[j], o.a[j][0], rx);
      ry = fmaf(Rj * is[j], o.a[j][1], ry);
      rz = fmaf(Rj * is[j], o.a[j][2], rz);
      tr += Q[j][j];
      dls[j] += -2.0f * Q[j][j];
    }
    const float z2 = 2.0f * iz;
    dX += z2 * rx;
    dY += z2 * ry;
    dZ += z2 * (tr + rz);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float q = -2.0f * o.s[k] * is[j] * Q[j][k];
#pragma unroll
        for (int m = 0; m < 3; ++m) dA[k][m] = fmaf(q, o.a[j][m], dA[k][m]);
      }
  } else {
    // Re-centred homography: c_k = P m_k (m_k = s_k a_k, P = [[1, 0, -x/z],
    // [0, 1, -y/z]]), E = [c_0 c_1], Q = Z E^-1 F^-1 and h = -m_z^T E^-1 F^-1
    // (F = diag(fx, fy)); a pixel has p = (Q xi, 1 + h xi), (u, v) = p / p_2.
    // The record gradient (slots 7-12) is A' = sum (du, dv) (u, v)^T and
    // b' = sum p_2 dL/dp_2 (u, v): with eta = E^-1 xi = (u, v) p_2 / Z,
    // dL/dE = -E^-T M for M = A' - m_z b'^T / Z, dL/dZ gains tr(A') / Z and
    // dL/dm_kz gains -b'_k / Z.  In the basis (a_0, a_1, n) of the splat,
    // dL/dm_k . a_j = -M_jk / s_j (j < 2) and dL/dm_k . n = -M_.k . E^-1 P n,
    // and dL/dlog s_k = -M_kk: E^-T never meets the thin axis's column, so a
    // needle-thin surfel's gradients keep binary32 accuracy.
    const float m0z = o.s[0] * o.a[0][2], m1z = o.s[1] * o.a[1][2];
    const float detE = det2(o.e0, o.e1, o.f0, o.f1);
    const float ie = 1.0f / detE;
    const float E00 = o.f1 * ie, E01 = -o.e1 * ie, E10 = -o.f0 * ie, E11 = o.e0 * ie;
    const bool ok = isfinite(ie) && isfinite(E00) && isfinite(E01) && isfinite(E10) && isfinite(E11);
    float dxz = dxc * fx, dyz = dyc * fy;
    if (ok) {
      const float bz0 = G[11] * iz, bz1 = G[12] * iz;
      dZ += (G[7] + G[10]) * iz;
      float M[2][2];
      M[0][0] = G[7] - m0z * bz0;
      M[0][1] = G[8] - m0z * bz1;
      M[1][0] = G[9] - m1z * bz0;
      M[1][1] = G[10] - m1z * bz1;
      const float pnx = o.a[2][0] - o.xz * o.a[2][2], pny = o.a[2][1] - o.yz * o.a[2][2];
      const float w0 = E00 * pnx + E01 * pny, w1 = E10 * pnx + E11 * pny;
      const float is0 = 1.0f / o.s[0], is1 = 1.0f / o.s[1];
      const float mz[2] = {m0z, m1z}, bz[2] = {bz0, bz1};
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float c0 = -M[0][k] * is0, c1 = -M[1][k] * is1, c2 = -(M[0][k] * w0 + M[1][k] * w1);
#pragma unroll
        for (int m = 0; m < 3; ++m) dA[k][m] += o.s[k] * (c0 * o.a[0][m] + c1 * o.a[1][m] + c2 * o.a[2][m]);
        // the h row: dL/dm_kz
        dA[k][2] += -o.s[k] * bz[k];
        dls[k] += -M[k][k] - o.s[k] * bz[k] * o.a[k][2];
        dxz += mz[k] * (E00 * M[0][k] + E10 * M[1][k]);
        dyz += mz[k] * (E01 * M[0][k] + E11 * M[1][k]);
      }
    }
    dX += dxz * iz;
    dY += dyz * iz;
    dZ += -(dxz * X + dyz * Y) * iz * iz;
    // scale modulation (Eqs. 6-7)
    float gate, fac;
    const float am = modulate(o.alpha, o.s[2], a.cfg, &gate, &fac);
    dalpha = G[0] * fac;
    const float dszs = G[0] * am * (-a.cfg.lambda_z);
    const float dsz = dszs * (gate + o.s[2] * gate * (1.f - gate) / a.cfg.T_z);
    dls[2] += dsz * o.s[2];
  }
  // projected centre (x_c = fx X/Z + cx) for 3D; 2D folded it into dxz above
  if (type == 1) {
    dX += dxc * fx * iz;
    dY += dyc * fy * iz;
    dZ += -(dxc * fx * X + dyc * fy * Y) * iz * iz;
  }
  // camera: mu_c = R_cw mu + t
  float dmu[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) dmu[k] = c.R[k] * dX + c.R[3 + k] * dY + c.R[6 + k] * dZ;
  // axes: a_k = R_cw Rq[:,k]  ->  dRq[:,k] = R_cw^T dA[k]
  float dR[9];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int r = 0; r < 3; ++r)
      dR[3 * r + k] = c.R[r] * dA[k][0] + c.R[3 + r] * dA[k][1] + c.R[6 + r] * dA[k][2];
  const float w = o.qn[0], x = o.qn[1], y = o.qn[2], z = o.qn[3];
  float dq[4];
  dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] - 2.f * x * dR[8]);
  dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] - 2.f * y * dR[8]);
  dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
  const float qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
  float4 gq;
  gq.x = (dq[0] - w * qd) * o.qinv;
  gq.y = (dq[1] - x * qd) * o.qinv;
  gq.z = (dq[2] - y * qd) * o.qinv;
  gq.w = (dq[3] - z * qd) * o.qinv;
  PGrad r;
  r.q = gq;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) r.dv[ch] = ctx.cpos[ch] ? G[1 + ch] : 0.0f;
  if (DEG > 0) {
    float wk[NB];
    ctx.visit_sh([&](int k, float f0, float f1, float f2) {
      wk[k] = r.dv[0] * f0 + r.dv[1] * f1 + r.dv[2] * f2;
    });
    float gd[3];
    sh_grad<DEG>(ctx.ux, ctx.uy, ctx.uz, wk, gd);
    const float dotp = gd[0] * ctx.ux + gd[1] * ctx.uy + gd[2] * ctx.uz;
    dmu[0] += (gd[0] - ctx.ux * dotp) * ctx.il;
    dmu[1] += (gd[1] - ctx.uy * dotp) * ctx.il;
    dmu[2] += (gd[2] - ctx.uz * dotp) * ctx.il;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.mu[k] = dmu[k];
    r.ls[k] = dls[k];
  }
  r.logit = dalpha * o.alpha * (1.f - o.alpha);
  return r;
}

__device__ __forceinline__ void load_rec_grad(const float *rec_grad, int64_t i, float (&G)[kGradW]) {
  const float4 *src = reinterpret_cast<const float4 *>(rec_grad) + 4 * i;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = src[k];
    G[4 * k] = v.x; G[4 * k + 1] = v.y; G[4 * k + 2] = v.z; G[4 * k + 3] = v.w;
  }
}

template <int DEG>
__device__ __forceinline__ void store_pgrad(const PrepGradArgs &g, int64_t i, const PGrad &r, const float *Yb) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    g.means[3 * i + k] = r.mu[k];
    g.log_scales[3 * i + k] = r.ls[k];
  }
  reinterpret_cast<float4 *>(g.quats)[i] = r.q;
  g.logits[i] = r.logit;
  float out[NB * 3];
#pragma unroll
  for (int k = 0; k < NB; ++k)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) out[3 * k + ch] = Yb ? r.dv[ch] * Yb[k] : 0.0f;
  store_sh<DEG>(g.sh + (int64_t)i * NB * 3, Yb ? out : nullptr);
}

template <int DEG>
__device__ __forceinline__ void store_zero_grad(const PrepGradArgs &g, int64_t i) {
  PGrad z;
#pragma unroll
  for (int k = 0; k < 3; ++k) { z.mu[k] = 0.f; z.ls[k] = 0.f; z.dv[k] = 0.f; }
  z.logit = 0.f;
  z.q = make_float4(0.f, 0.f, 0.f, 0.f);
  store_pgrad<DEG>(g, i, z, nullptr);
}

// The SH gradient rows of a warp's 32 primitives are contiguous: where a row
// is a whole number of 16-byte words (degrees 1 and 3) the warp stages 16
// rows at a time in shared memory and writes them as one contiguous run, so
// every store covers whole lines instead of 32 partial sectors.
template <int DEG>
__device__ __forceinline__ void store_sh_rows_warp(float *sh, int64_t n, int64_t i, const float *v,
                                                   float4 *stage) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
  constexpr int RW = NB * 3 / 4;  // float4 words per row
  const int lane = threadIdx.x & 31;
  const int64_t i0 = i - lane;
  float4 *dst = reinterpret_cast<float4 *>(sh);
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    if ((lane >> 4) == half) {
      float4 *row = stage + (lane & 15) * RW;
#pragma unroll
      for (int k = 0; k < RW; ++k)
        row[k] = v ? make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3])
                   : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    const int64_t r0 = i0 + 16 * half;
    const int64_t left = n - r0;
    const int words = left <= 0 ? 0 : (int)(left < 16 ? left : 16) * RW;
    for (int k = lane; k < words; k += 32) dst[r0 * RW + k] = stage[k];
    __syncwarp();
  }
}

template <int DEG>
__global__ void __launch_bounds__(256, 3) preprocess_bwd_kernel(PrepArgs a, PrepGradArgs g) {
  grid_dep();
  constexpr int NB = (DEG + 1) * (DEG + 1);
  constexpr bool kWarpRows = DEG == 1 || DEG == 3;
  __shared__ float4 stage[kWarpRows ? 8 : 1][kWarpRows ? 16 * NB * 3 / 4 : 1];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = i < a.n;
  const bool binned = in && __ldg(a.touched + i) != 0u;
  PGrad r;
  float out[NB * 3];
  if (binned) {
    // the SH row and the record gradient are read after the contract's
    // arithmetic: ask L2 for them first (a hint only)
    if constexpr (NB > 1) {
      const char *sp = reinterpret_cast<const char *>(a.sh + i * NB * 3);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(sp));
      if (NB * 12 > 96) asm volatile("prefetch.global.L2 [%0];" ::"l"(sp + 96));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(sp + NB * 12 - 4));
    }
    asm volatile("prefetch.global.L2 [%0];" ::"l"(g.rec_grad + i * kGradW));
    BwdCtx<DEG, true> x;
    bwd_ctx<DEG, true>(a, i, x);
    float G[kGradW];
    load_rec_grad(g.rec_grad, i, G);
    r = chain_grad<DEG, true>(a, x, G);
#pragma unroll
    for (int k = 0; k < NB; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) out[3 * k + ch] = r.dv[ch] * x.Yb[k];
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) { r.mu[k] = 0.f; r.ls[k] = 0.f; r.dv[k] = 0.f; }
    r.logit = 0.f;
    r.q = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (in) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      g.means[3 * i + k] = r.mu[k];
      g.log_scales[3 * i + k] = r.ls[k];
    }
    reinterpret_cast<float4 *>(g.quats)[i] = r.q;
    g.logits[i] = r.logit;
  }
  if constexpr (kWarpRows) {
    store_sh_rows_warp<DEG>(g.sh, a.n, i, binned ? out : nullptr, stage[threadIdx.x >> 5]);
  } else {
    if (in) store_sh<DEG>(g.sh + i * NB * 3, binned ? out : nullptr);
  }
}


// Frequency-decoupled optimisation, Algorithm 1 (§3.3): with g_low and
// g_high the primitive's full raw-parameter gradients (means, log-scales,
// quaternion, opacity logit and all SH coefficients, concatenated) from the
// low- and high-frequency losses, a conflict is g_low . g_high < 0.  Then a
// surfel (t = 0) keeps g_low and replaces g_high by its component normal to
// g_low (Eq. 9); a 3D Gaussian keeps g_high and projects g_low (Eq. 10).  The
// update is g_color + g_low + g_high.  Each gradient is the linear chain of
// its record gradient, so the three are formed in registers and only the
// sum is written.  The SH block of each gradient is dv (x) Y, so its dot
// products are (dv . dv') |Y|^2.
__device__ __forceinline__ float pgrad_dot(const PGrad &p, const PGrad &q, float yy) {
  float d = p.logit * q.logit + p.q.x * q.q.x + p.q.y * q.q.y + p.q.z * q.q.z + p.q.w * q.q.w;
#pragma unroll
  for (int k = 0; k < 3; ++k) d += p.mu[k] * q.mu[k] + p.ls[k] * q.ls[k] + yy * p.dv[k] * q.dv[k];
  return d;
}

__device__ __forceinline__ void pgrad_axpy(PGrad &y, float s, const PGrad &x) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    y.mu[k] = fmaf(s, x.mu[k], y.mu[k]);
    y.ls[k] = fmaf(s, x.ls[k], y.ls[k]);
    y.dv[k] = fmaf(s, x.dv[k], y.dv[k]);
  }
  y.logit = fmaf(s, x.logit, y.logit);
  y.q.x = fmaf(s, x.q.x, y.q.x); y.q.y = fmaf(s, x.q.y, y.q.y);
  y.q.z = fmaf(s, x.q.z, y.q.z); y.q.w = fmaf(s, x.q.w, y.q.w);
}

template <int DEG>
__global__ void __launch_bounds__(128) preprocess_bwd_fdo_kernel(PrepArgs a, PrepGradFdoArgs g3) {
  grid_dep();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  PrepGradArgs g;
  g.rec_grad = nullptr;
  g.means = g3.means; g.log_scales = g3.log_scales; g.quats = g3.quats; g.logits = g3.logits; g.sh = g3.sh;
  if (__ldg(a.touched + i) == 0u) {
    store_zero_grad<DEG>(g, i);
    return;
  }
  BwdCtx<DEG, false> x;
  bwd_ctx<DEG, false>(a, i, x);
  float yy = 0.0f;
#pragma unroll
  for (int k = 0; k < BwdCtx<DEG, false>::NB; ++k) yy = fmaf(x.Yb[k], x.Yb[k], yy);
  float G[kGradW];
  load_rec_grad(g3.rec_low, i, G);
  PGrad pl = chain_grad<DEG, false>(a, x, G);
  load_rec_grad(g3.rec_high, i, G);
  PGrad ph = chain_grad<DEG, false>(a, x, G);
  const float lh = pgrad_dot(pl, ph, yy);
  if (lh < 0.0f) {
    if (x.type == 0) {
      pgrad_axpy(ph, -lh / pgrad_dot(pl, pl, yy), pl);  // Eq. 9
    } else {
      pgrad_axpy(pl, -lh / pgrad_dot(ph, ph, yy), ph);  // Eq. 10
    }
    if (g3.n_conflicts) atomicAdd(g3.n_conflicts, 1ull);
  }
  load_rec_grad(g3.rec_color, i, G);
  PGrad r = chain_grad<DEG, false>(a, x, G);
  pgrad_axpy(r, 1.0f, pl);
  pgrad_axpy(r, 1.0f, ph);
  store_pgrad<DEG>(g, i, r, x.Yb);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int launch_preprocess_fwd(const PrepArgs &a, int deg, cudaStream_t s) {
  if (a.n == 0) return 0;
  const unsigned grid = (unsigned)((a.n + 255) / 256);
  switch (deg) {
    case 0: preprocess_fwd_kernel<0><<<grid, 256, 0, s>>>(a); break;
    case 1: preprocess_fwd_kernel<1><<<grid, 256, 0, s>>>(a); break;
    case 2: preprocess_fwd_kernel<2><<<grid, 256, 0, s>>>(a); break;
    default: preprocess_fwd_kernel<3><<<grid, 256, 0, s>>>(a); break;
  }
  return 0;
}

int launch_preprocess_batch(const BatchPrepArgs &b, cudaStream_t s) {
  const int64_t total = b.base[b.nreq];
  if (total == 0) return 0;
  preprocess_batch_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(b);
  return 0;
}

int launch_preprocess_bwd(const PrepArgs &a, const PrepGradArgs &g, int deg, cudaStream_t s) {
  if (a.n == 0) return 0;
  const unsigned grid = (unsigned)((a.n + 255) / 256);
  switch (deg) {
    case 0: pdl_launch(preprocess_bwd_kernel<0>, grid, 256, 0, s, a, g); break;
    case 1: pdl_launch(preprocess_bwd_kernel<1>, grid, 256, 0, s, a, g); break;
    case 2: pdl_launch(preprocess_bwd_kernel<2>, grid, 256, 0, s, a, g); break;
    default: pdl_launch(preprocess_bwd_kernel<3>, grid, 256, 0, s, a, g); break;
  }
  return 0;
}

int launch_preprocess_bwd_fdo(const PrepArgs &a, const PrepGradFdoArgs &g, int deg, cudaStream_t s) {
  if (a.n == 0) return 0;
  const unsigned grid = (unsigned)((a.n + 127) / 128);
  switch (deg) {
    case 0: pdl_launch(preprocess_bwd_fdo_kernel<0>, grid, 128, 0, s, a, g); break;
    case 1: pdl_launch(preprocess_bwd_fdo_kernel<1>, grid, 128, 0, s, a, g); break;
    case 2: pdl_launch(preprocess_bwd_fdo_kernel<2>, grid, 128, 0, s, a, g); break;
    default: pdl_launch(preprocess_bwd_fdo_kernel<3>, grid, 128, 0, s, a, g); break;
  }
  return 0;
}

}  // namespace hgs
