"""Pins of the training-loop oracle: Adam against its closed form at step 1
and against torch.optim.Adam over several steps (float64), the
densification rules on hand-built primitives, the geometry of split samples
(exact offsets for unit draws, covariance for many draws) and the opacity
reset."""
import numpy as np
import pytest
import torch

from oracle import train as T


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(0)
    p, g = rng.normal(size=50), rng.normal(size=50)
    p2, m2, v2 = T.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(p2, p - 1e-3 * np.sign(g), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m2, 0.1 * g)
    np.testing.assert_allclose(v2, 0.001 * g * g)


def test_adam_matches_torch_over_steps():
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=200)
    grads = rng.normal(size=(6, 200))
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=5e-3, betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0.copy(), np.zeros(200), np.zeros(200)
    for k in range(6):
        opt.zero_grad()
        t.grad = torch.tensor(grads[k], dtype=torch.float64)
        opt.step()
        p, m, v = T.adam_step(p, grads[k], m, v, k + 1, lr=5e-3)
    np.testing.assert_allclose(p, t.detach().numpy(), rtol=0, atol=1e-13)


def _prims():
    # A hot+small, B hot+big, C cold+transparent, D cold+opaque, E never seen,
    # F surfel hot whose in-plane scales are small (sentinel s_z ignored)
    ls = np.log(np.array([[0.01, 0.01, 0.01], [0.2, 0.05, 0.05], [0.01] * 3, [0.01] * 3, [0.01] * 3,
                          [0.02, 0.01, 1e-13]]))
    logits = np.array([1.0, 1.0, -8.0, 2.0, 2.0, 1.0])
    types = np.array([1, 1, 1, 1, 1, 0], np.uint8)
    acc = np.array([3e-3, 3e-3, 0.0, 1e-5, 0.0, 9e-3])
    cnt = np.array([3, 3, 2, 2, 0, 3])
    return ls, logits, types, acc, cnt


def test_densify_actions_hand_built():
    ls, logits, types, acc, cnt = _prims()
    a = T.densify_actions(acc, cnt, ls, logits, types, grad_thresh=2e-4, size_thresh=0.1, min_opacity=0.005)
    assert list(a) == [2, 3, 0, 1, 1, 2]


def test_densify_outputs_and_split_geometry():
    ls, logits, types, acc, cnt = _prims()
    n = len(types)
    rng = np.random.default_rng(2)
    q = rng.normal(size=(n, 4))
    params = {"means": rng.normal(size=(n, 3)), "log_scales": ls, "quats": q, "opacity_logits": logits,
              "sh": rng.normal(size=(n, 16, 3))}
    moments = {"m_means": rng.normal(size=(n, 3))}
    z = np.zeros((n, 2, 3))
    z[1, 0] = [1.0, 0.0, 0.0]      # first sample of B moves one scale along its first axis
    z[1, 1] = [0.0, 0.0, 0.0]
    out, tout, mom, act = T.densify(params, types, moments, acc, cnt, z, 2e-4, 0.1, 0.005)
    # A, A', B1, B2, D, E, F, F'
    assert len(tout) == 8
    np.testing.assert_array_equal(out["means"][0], params["means"][0])
    np.testing.assert_array_equal(out["means"][1], params["means"][0])
    np.testing.assert_array_equal(mom["m_means"][0], moments["m_means"][0])
    np.testing.assert_array_equal(mom["m_means"][1], 0.0)
    R = T.quat_to_rot(q[1])
    np.testing.assert_allclose(out["means"][2], params["means"][1] + 0.2 * R[:, 0], atol=1e-14)
    np.testing.assert_allclose(out["means"][3], params["means"][1], atol=1e-14)
    np.testing.assert_allclose(out["log_scales"][2], ls[1] - np.log(1.6), atol=1e-14)
    np.testing.assert_array_equal(mom["m_means"][2:4], 0.0)
    np.testing.assert_array_equal(out["sh"][2], params["sh"][1])
    assert list(tout) == [1, 1, 1, 1, 1, 1, 0, 0]


def test_split_samples_follow_the_covariance():
    n = 1
    ls = np.log(np.array([[0.3, 0.1, 0.05]]))
    rng = np.random.default_rng(3)
    q = rng.normal(size=(1, 4))
    R = T.quat_to_rot(q[0])
    draws = rng.normal(size=(6000, 3))
    pts = []
    for k in range(0, 6000, 2):
        params = {"means": np.zeros((1, 3)), "log_scales": ls, "quats": q, "opacity_logits": np.array([1.0]),
                  "sh": np.zeros((1, 1, 3))}
        out, *_ = T.densify(params, np.array([1], np.uint8), {}, np.array([1.0]), np.array([1]),
                            draws[k:k + 2][None], 1e-4, 0.0, 0.005)
        pts.append(out["means"])
    pts = np.concatenate(pts)
    cov = np.cov(pts.T)
    ref = R @ np.diag(np.exp(2 * ls[0])) @ R.T
    np.testing.assert_allclose(cov, ref, atol=0.06 * ref.max())


def test_reset_opacity_caps_alpha():
    lg = np.array([-9.0, -4.0, 0.0, 5.0])
    out = T.reset_opacity(lg, 0.01)
    alpha = 1 / (1 + np.exp(-out))
    assert np.all(alpha <= 0.01 + 1e-15)
    cap = np.log(0.01 / 0.99)                  # = -4.595: alpha 0.018 at -4 is capped
    assert out[0] == -9.0 and out[1] == pytest.approx(cap) and out[2] == pytest.approx(cap)
