"""Pins of the training-step oracle (loss, SSIM, Adam, compaction) against
closed forms, an independent library evaluation and finite differences."""
import numpy as np
import pytest

from oracle import train as T


def test_window_is_normalised_gaussian():
    w = T.gaussian_window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])
    r = np.arange(11) - 5.0
    g = np.exp(-r * r / 4.5)
    assert np.allclose(w, np.outer(g, g) / g.sum() ** 2, rtol=1e-14, atol=0)


def test_window_sum_matches_scipy():
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    img = rng.standard_normal((23, 31))
    w = T.gaussian_window()
    ref = nd.correlate(img, w, mode="constant", cval=0.0)
    assert np.allclose(T.window_sum(img, w), ref, rtol=0, atol=1e-13)
    # an asymmetric window catches a flipped (convolution) orientation
    wa = rng.random((11, 11))
    assert np.allclose(T.window_sum(img, wa), nd.correlate(img, wa, mode="constant", cval=0.0), rtol=0, atol=1e-12)


def test_ssim_identity_and_constant_closed_form():
    rng = np.random.default_rng(1)
    x = rng.random((3, 20, 24))
    assert np.allclose(T.ssim_map(x, x), 1.0, rtol=0, atol=1e-12)
    a, b = 0.3, 0.7
    s = T.ssim_map(np.full((1, 30, 30), a), np.full((1, 30, 30), b))
    inner = s[0, 5:-5, 5:-5]
    closed = (2 * a * b + T.SSIM_C1) / (a * a + b * b + T.SSIM_C1)
    assert np.allclose(inner, closed, rtol=0, atol=1e-12)
    # at the border the zero padding lowers both means by the same factor k:
    # ssim = (2 k^2 ab + C1)(2 cov + C2) / ((k^2 (a^2+b^2) + C1)(var_x + var_y + C2))
    k = T.gaussian_window()[5:, :].sum()          # window mass inside at a top-edge pixel
    mx, my = k * a, k * b
    vx, vy, cxy = k * a * a - mx * mx, k * b * b - my * my, k * a * b - mx * my
    edge = ((2 * mx * my + T.SSIM_C1) * (2 * cxy + T.SSIM_C2)) / ((mx * mx + my * my + T.SSIM_C1) * (vx + vy + T.SSIM_C2))
    assert abs(s[0, 0, 15] - edge) < 1e-12


def test_loss_definition_pieces():
    rng = np.random.default_rng(2)
    X = rng.random((3, 16, 18))
    Ct = rng.random((3, 16, 18)) * 0.5
    At = rng.random((16, 18))
    A = rng.random((16, 18))
    bg = (0.2, 0.4, 0.9)
    Y = Ct + (1 - At)[None] * np.array(bg).reshape(3, 1, 1)
    L = T.loss(X, A, Ct, At, bg, 0.2, 0.5)
    ref = 0.8 * np.abs(X - Y).mean() + 0.2 * (1 - T.ssim_map(X, Y).mean()) + 0.5 * np.abs(A - At).mean()
    assert abs(L - ref) < 1e-14
    assert abs(T.loss_grad(X, A, Ct, At, bg, 0.2, 0.5)[0] - L) < 1e-13
    # identical images and alpha: zero loss
    assert abs(T.loss(Y, At, Ct, At, bg, 0.2, 0.5)) < 1e-12


@pytest.mark.parametrize("lam,w_alpha", [(0.2, 0.0), (0.2, 0.7), (1.0, 0.0)])
def test_loss_gradient_finite_differences(lam, w_alpha):
    rng = np.random.default_rng(3)
    H, W = 14, 17
    X = rng.random((3, H, W))
    A = rng.random((H, W))
    Ct = rng.random((3, H, W)) * 0.6
    At = rng.random((H, W))
    bg = (0.1, 0.5, 0.3)
    _, gi, ga = T.loss_grad(X, A, Ct, At, bg, lam, w_alpha)
    h = 1e-6
    for (c, y, x) in [(0, 0, 0), (1, 7, 8), (2, 13, 16), (0, 3, 15), (1, 12, 1), (2, 6, 0)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[c, y, x] += h
        Xm[c, y, x] -= h
        fd = (T.loss(Xp, A, Ct, At, bg, lam, w_alpha) - T.loss(Xm, A, Ct, At, bg, lam, w_alpha)) / (2 * h)
        assert abs(fd - gi[c, y, x]) < 1e-8 + 1e-5 * abs(fd), (c, y, x, fd, gi[c, y, x])
    for (y, x) in [(0, 0), (5, 9), (13, 16)]:
        Ap, Am = A.copy(), A.copy()
        Ap[y, x] += h
        Am[y, x] -= h
        fd = (T.loss(X, Ap, Ct, At, bg, lam, w_alpha) - T.loss(X, Am, Ct, At, bg, lam, w_alpha)) / (2 * h)
        assert abs(fd - ga[y, x]) < 1e-9, (y, x, fd, ga[y, x])


def test_adam_constant_gradient_closed_form():
    rng = np.random.default_rng(4)
    p0 = rng.standard_normal((5, 3))
    g = rng.standard_normal((5, 3))
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    lr = 0.01
    for t in range(1, 8):
        p, m, v = T.adam_step(p, g, m, v, t, lr)
        # bias-corrected moments of a constant gradient are g and g^2
        assert np.allclose(p, p0 - t * lr * np.sign(g), rtol=0, atol=1e-12)
    # first step by hand, with a visible epsilon
    p1, m1, v1 = T.adam_step(p0, g, np.zeros_like(p0), np.zeros_like(p0), 1, lr, eps=1e-3)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    assert np.allclose(p1, p0 - lr * g / (np.abs(g) + 1e-3), rtol=0, atol=1e-15)


def test_adam_frozen_rows_untouched():
    rng = np.random.default_rng(5)
    p0 = rng.standard_normal((6, 4, 3))
    g = rng.standard_normal((6, 4, 3))
    m0 = rng.standard_normal((6, 4, 3)) * 0.1
    v0 = rng.random((6, 4, 3)) * 0.1
    fr = np.array([0, 1, 0, 0, 1, 0], bool)
    p, m, v = T.adam_step(p0, g, m0, v0, 3, 0.05, frozen_rows=fr)
    assert np.array_equal(p[fr], p0[fr]) and np.array_equal(m[fr], m0[fr]) and np.array_equal(v[fr], v0[fr])
    assert np.all(p[~fr] != p0[~fr])


def test_compact_keeps_order():
    a = np.arange(20).reshape(10, 2)
    keep = np.array([1, 0, 0, 1, 1, 0, 1, 0, 0, 1], bool)
    assert np.array_equal(T.compact(a, keep), a[[0, 3, 4, 6, 9]])


def _golden(name):
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_activity_weights_are_the_papers():
    g = _golden("inactive_pruning.txt")
    assert T.ACT_W == (g["w_p"], g["w_c"], g["w_s"])


def test_activity_constant_gradient_closed_form():
    """With a constant gradient every Adam update is lr sign(g) per element, so
    the step's norms are lr sqrt(elements) and the sample is their weighted sum."""
    rng = np.random.default_rng(6)
    n, K = 7, 16
    lr = (1.6e-4, 2.5e-3, 5e-3)            # means, SH, log-scales
    shapes = [(n, 3), (n, K, 3), (n, 3)]
    p = [rng.standard_normal(s) for s in shapes]
    g = [rng.standard_normal(s) for s in shapes]
    m = [np.zeros(s) for s in shapes]
    v = [np.zeros(s) for s in shapes]
    acc = np.zeros(n)
    for t in range(1, 6):
        d = []
        for k in range(3):
            p1, m[k], v[k] = T.adam_step(p[k], g[k], m[k], v[k], t, lr[k])
            d.append(p1 - p[k])
            p[k] = p1
        acc += T.activity_sample(*d)
    per_step = 2 * lr[0] * np.sqrt(3) + 0.1 * lr[1] * np.sqrt(3 * K) + 0.1 * lr[2] * np.sqrt(3)
    assert np.allclose(acc, 5 * per_step, rtol=1e-9)


def test_activity_prune_threshold_and_decay():
    g = _golden("inactive_pruning.txt")
    dR, T0, decay = int(g["dR"]), g["T0"], g["decay"]
    acc = np.array([0.5, 1.5, 1.4999, 0.0, 3.0]) * dR * 0.01     # averages 0.005, 0.015, 0.014999, 0, 0.03
    trainable = np.array([1, 1, 1, 0, 1], bool)
    keep = T.activity_prune(acc, dR, T0, trainable)
    # <= T0 removed (equality included), frozen rows never tested
    assert keep.tolist() == [False, False, False, True, True]
    # the threshold after k comparisons is T0 * decay^k
    thr = T0
    for _ in range(10):
        thr *= decay
    assert abs(thr - 0.015 * 0.975 ** 10) < 1e-15
