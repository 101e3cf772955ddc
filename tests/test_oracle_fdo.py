"""Pins of the frequency-decoupled-optimisation oracle (EGGS §3.3, Eq. 8,
Algorithm 1; App. E) against facts fixed by the mathematics: orthogonality
and perfect reconstruction of the Haar transform, Parseval, band patterns
of constant / striped / checkered images, a hand-computed 2x2 example,
finite differences, and the projection's geometry on worked examples."""
import numpy as np
import pytest

from oracle import fdo as F


@pytest.mark.parametrize("n", [2, 4, 10])
def test_haar_analysis_is_orthogonal(n):
    L, H = F.haar_matrices(n)
    Q = np.vstack([L, H])
    np.testing.assert_allclose(Q @ Q.T, np.eye(n), atol=1e-15)
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), atol=1e-15)


def test_perfect_reconstruction_and_parseval():
    rng = np.random.default_rng(0)
    img = rng.normal(size=(3, 6, 8))
    b = F.dwt_bands(img)
    Lr, Hr = F.haar_matrices(6)
    Lc, Hc = F.haar_matrices(8)
    rec = Lr.T @ b["LL"] @ Lc + Hr.T @ b["LH"] @ Lc + Lr.T @ b["HL"] @ Hc + Hr.T @ b["HH"] @ Hc
    np.testing.assert_allclose(rec, img, atol=1e-13)
    energy = sum((v ** 2).sum() for v in b.values())
    assert abs(energy - (img ** 2).sum()) < 1e-10


def test_band_patterns():
    H, W = 6, 8
    y, x = np.mgrid[0:H, 0:W]
    const = np.full((1, H, W), 0.7)
    b = F.dwt_bands(const)
    np.testing.assert_allclose(b["LL"], 1.4, atol=1e-14)  # 4 * 0.7 / 2
    for k in ("LH", "HL", "HH"):
        np.testing.assert_allclose(b[k], 0.0, atol=1e-14)
    rows = ((-1.0) ** y)[None]           # alternates down the rows
    cols = ((-1.0) ** x)[None]           # alternates along the columns
    checker = ((-1.0) ** (x + y))[None]
    for img, live in ((rows, "LH"), (cols, "HL"), (checker, "HH")):
        b = F.dwt_bands(img)
        for k, v in b.items():
            np.testing.assert_allclose(v, 2.0 if k == live else 0.0, atol=1e-14)


def test_hand_computed_2x2():
    img = np.array([[[1.0, 2.0], [3.0, 4.0]]])
    b = F.dwt_bands(img)
    assert b["LL"][0, 0, 0] == pytest.approx(5.0)
    assert b["LH"][0, 0, 0] == pytest.approx(-2.0)
    assert b["HL"][0, 0, 0] == pytest.approx(-1.0)
    assert b["HH"][0, 0, 0] == pytest.approx(0.0, abs=1e-15)
    l1, low, high = F.image_losses(img, np.zeros_like(img))
    assert l1 == pytest.approx(2.5)
    assert low == pytest.approx(25.0)
    assert high == pytest.approx(5.0 / 3.0)


@pytest.mark.parametrize("shape", [(3, 6, 8), (2, 5, 7), (1, 7, 4)])
def test_loss_gradients_match_finite_differences(shape):
    rng = np.random.default_rng(1)
    img = rng.normal(size=shape)
    tgt = rng.normal(size=shape)
    w = (0.7, 0.2, 0.4)
    g = F.loss_grads(img, tgt, w)
    h = 1e-6
    for _ in range(12):
        idx = tuple(int(rng.integers(s)) for s in shape)
        p, m = img.copy(), img.copy()
        p[idx] += h
        m[idx] -= h
        lp, lm = F.image_losses(p, tgt), F.image_losses(m, tgt)
        for k in range(3):
            fd = w[k] * (lp[k] - lm[k]) / (2 * h)
            assert g[k][idx] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # the odd border is outside the DWT: no frequency gradient there
    if shape[2] % 2:
        assert np.all(g[1][:, :, -1] == 0) and np.all(g[2][:, :, -1] == 0)
    if shape[1] % 2:
        assert np.all(g[1][:, -1, :] == 0) and np.all(g[2][:, -1, :] == 0)


def _one(v):
    return {"means": np.asarray(v, float)[None, :3], "log_scales": np.zeros((1, 3)),
            "quats": np.zeros((1, 4)), "opacity_logits": np.zeros(1), "sh": np.zeros((1, 1, 3))}


def test_algorithm1_worked_examples():
    gc, gl, gh = _one([0.0, 0.0, 1.0]), _one([1.0, 0.0, 0.0]), _one([-1.0, 1.0, 0.0])
    # surfel: keep g_low, g_high loses its component along g_low (Eq. 9)
    out, conf, _ = F.algorithm1(gc, gl, gh, [0])
    assert conf[0]
    np.testing.assert_allclose(out["means"][0], [1.0, 1.0, 1.0])    # (0,0,1) + (1,0,0) + (0,1,0)
    # 3D Gaussian: keep g_high, g_low loses its component along g_high (Eq. 10)
    out, conf, _ = F.algorithm1(gc, gl, gh, [1])
    assert conf[0]
    np.testing.assert_allclose(out["means"][0], [-0.5, 1.5, 1.0])   # (0,0,1) + (0.5,0.5,0) + (-1,1,0)
    # no conflict: plain sum
    out, conf, _ = F.algorithm1(gc, gl, _one([1.0, 1.0, 0.0]), [0])
    assert not conf[0]
    np.testing.assert_allclose(out["means"][0], [2.0, 1.0, 1.0])


def test_algorithm1_projection_geometry():
    rng = np.random.default_rng(2)
    n = 40
    def rnd():
        return {"means": rng.normal(size=(n, 3)), "log_scales": rng.normal(size=(n, 3)),
                "quats": rng.normal(size=(n, 4)), "opacity_logits": rng.normal(size=n),
                "sh": rng.normal(size=(n, 16, 3))}
    gc, gl, gh = rnd(), rnd(), rnd()
    zero = {k: np.zeros_like(v) for k, v in gc.items()}
    types = rng.integers(0, 2, n)
    out, conf, _ = F.algorithm1(zero, gl, gh, types)
    for i in range(n):
        l, h, u = F.flatten(gl, i), F.flatten(gh, i), F.flatten(out, i)
        if not conf[i]:
            np.testing.assert_allclose(u, l + h, atol=1e-12)
        elif types[i] == 0:          # u = g_low + g_high', g_high' orthogonal to g_low
            assert abs((u - l) @ l) < 1e-9 * (l @ l)
        else:                        # u = g_low' + g_high, g_low' orthogonal to g_high
            assert abs((u - h) @ h) < 1e-9 * (h @ h)
    assert 0 < conf.sum() < n
    # the appearance gradient passes straight through
    out2, _, _ = F.algorithm1(gc, gl, gh, types)
    for k in gc:
        np.testing.assert_allclose(out2[k] - out[k], gc[k], atol=1e-12)
