"""FP64 oracle of the training step around the rasterizer: the image loss and
its gradient, Adam, and the compaction that applies a prune.

TEST INFRASTRUCTURE.  Same rule as the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the oracle legs of ``bench.py`` may import it.
Plain numpy in double precision, written from the definitions below; no code
is shared with ``paper_2410_16978_gb300``.

Definitions (Sec. 3.2: each layer is optimised with the layers below it
frozen, a random background colour per frame and the alpha channel in the
loss; the image loss is that of the 3DGS training the paper builds on):

* target under background bg: Y = C_t + (1 - A_t) bg, with C_t the target's
  premultiplied colour and A_t its alpha.
* SSIM (Wang et al. 2004) per channel with an 11x11 Gaussian window of
  sigma 1.5 (normalised), zero padding outside the image, C1 = 0.01^2,
  C2 = 0.03^2:  mu_x = G*x, sx = G*(x^2) - mu_x^2, sxy = G*(xy) - mu_x mu_y,
  ssim = (2 mu_x mu_y + C1)(2 sxy + C2) / ((mu_x^2 + mu_y^2 + C1)(sx + sy + C2)),
  averaged over channels and pixels.
* loss = (1 - lam) mean|X - Y| + lam (1 - SSIM(X, Y)) + w_a mean|A - A_t|
  with lam = 0.2 (reading of "L1 + 0.2 D-SSIM" as the 3DGS weighting) and
  w_a the alpha weight (reading: an L1 term on alpha; the paper gives no form).
* Adam (Kingma & Ba 2015) with bias correction, one learning rate per
  parameter group; Gaussians of frozen layers keep parameters and moments.

* Inactive pruning (Sec. 3.2.2): per trainable Gaussian and step i, p_i, c_i,
  s_i are the Euclidean norms of the update Adam applied to its mean, its SH
  coefficients (colour) and its log-scales; AvgSample = (1/dR) sum over dR
  steps of (2 p_i + 0.1 c_i + 0.1 s_i); a trainable Gaussian is removed when
  AvgSample <= T, and T is multiplied by 0.975 after each comparison (T0 =
  0.015, dR = 100).  Reading: "norm" is the norm of the per-step update (the
  activity of the optimisation), colour is every SH coefficient, scale is the
  stored log-scale; Gaussians of frozen layers are not tested.

Parity status: activity pinned by the constant-gradient closed form (each
update is lr sign(g), so the norms are lr sqrt(count)) and the paper's
constants (tests/golden/inactive_pruning.txt); ssim / loss pinned by SSIM(x, x) = 1, the interior closed form
for constant images, an independent scipy.ndimage evaluation of the window
sums, and central finite differences of the loss; adam pinned by the
constant-gradient closed form (each step moves by lr sign(g)) and a
hand-computed first step; compact pinned by its definition on small arrays.
"""
from __future__ import annotations

import numpy as np

SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
SSIM_WIN = 11
SSIM_SIGMA = 1.5


def gaussian_window(size: int = SSIM_WIN, sigma: float = SSIM_SIGMA) -> np.ndarray:
    """Normalised 2-D Gaussian window, the outer product of the 1-D one."""
    r = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(r * r) / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def window_sum(img: np.ndarray, win: np.ndarray) -> np.ndarray:
    """out[y, x] = sum_{i, j} win[i, j] img[y + i - h, x + j - h], zero outside
    the image (h = half window); written as an explicit sum of shifted copies."""
    h = win.shape[0] // 2
    H, W = img.shape
    pad = np.zeros((H + 2 * h, W + 2 * h))
    pad[h:h + H, h:h + W] = img
    out = np.zeros((H, W))
    for i in range(win.shape[0]):
        for j in range(win.shape[1]):
            out += win[i, j] * pad[i:i + H, j:j + W]
    return out


def _moments(x, y, win):
    mx, my = window_sum(x, win), window_sum(y, win)
    sx = window_sum(x * x, win) - mx * mx
    sy = window_sum(y * y, win) - my * my
    sxy = window_sum(x * y, win) - mx * my
    return mx, my, sx, sy, sxy


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-pixel SSIM of two [C, H, W] images, channel by channel."""
    win = gaussian_window()
    out = np.zeros(x.shape)
    for c in range(x.shape[0]):
        mx, my, sx, sy, sxy = _moments(np.asarray(x[c], np.float64), np.asarray(y[c], np.float64), win)
        out[c] = ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sx + sy + SSIM_C2))
    return out


def target_under(bg, target_rgb, target_alpha) -> np.ndarray:
    """Y = C_t + (1 - A_t) bg."""
    bg = np.asarray(bg, np.float64).reshape(3, 1, 1)
    return np.asarray(target_rgb, np.float64) + (1.0 - np.asarray(target_alpha, np.float64))[None] * bg


def loss(image, alpha, target_rgb, target_alpha, bg, lam: float = 0.2, w_alpha: float = 0.0) -> float:
    X = np.asarray(image, np.float64)
    Y = target_under(bg, target_rgb, target_alpha)
    l1 = np.abs(X - Y).mean()
    s = ssim_map(X, Y).mean()
    la = np.abs(np.asarray(alpha, np.float64) - np.asarray(target_alpha, np.float64)).mean() if w_alpha else 0.0
    return (1.0 - lam) * l1 + lam * (1.0 - s) + w_alpha * la


def loss_grad(image, alpha, target_rgb, target_alpha, bg, lam: float = 0.2, w_alpha: float = 0.0):
    """(loss, dL/dimage [3,H,W], dL/dalpha [H,W]).  With f = ssim(mu_x, mu_y,
    sx, sy, sxy) per pixel q and G symmetric,
      d SSIM / d x_p = sum_q G(p - q) [df/dmu_x - 2 mu_x df/dsx - mu_y df/dsxy
                                       + 2 x_p df/dsx + y_p df/dsxy]_q
    i.e. three window sums of per-pixel maps.  |.|' is sign(.), 0 at 0."""
    X = np.asarray(image, np.float64)
    Y = target_under(bg, target_rgb, target_alpha)
    C, H, W = X.shape
    n = C * H * W
    win = gaussian_window()
    d_img = (1.0 - lam) * np.sign(X - Y) / n
    ssum = 0.0
    for c in range(C):
        x, y = X[c], Y[c]
        mx, my, sx, sy, sxy = _moments(x, y, win)
        n1 = 2 * mx * my + SSIM_C1
        n2 = 2 * sxy + SSIM_C2
        d1 = mx * mx + my * my + SSIM_C1
        d2 = sx + sy + SSIM_C2
        f = n1 * n2 / (d1 * d2)
        ssum += f.sum()
        df_dmx = f * (2 * my / n1 - 2 * mx / d1)
        df_dsx = -f / d2
        df_dsxy = 2 * f / n2
        a = df_dmx - 2 * mx * df_dsx - my * df_dsxy
        dS = window_sum(a, win) + 2 * x * window_sum(df_dsx, win) + y * window_sum(df_dsxy, win)
        d_img[c] += -lam * dS / n
    A = np.asarray(alpha, np.float64)
    At = np.asarray(target_alpha, np.float64)
    d_al = w_alpha * np.sign(A - At) / (H * W) if w_alpha else np.zeros((H, W))
    L = (1.0 - lam) * np.abs(X - Y).mean() + lam * (1.0 - ssum / n) + (w_alpha * np.abs(A - At).mean() if w_alpha else 0.0)
    return L, d_img, d_al


def adam_step(param, grad, m, v, t: int, lr: float, frozen_rows=None, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step on float64 copies; rows (first axis = Gaussian) marked in
    frozen_rows keep param, m and v.  Returns (param, m, v)."""
    p = np.array(param, np.float64)
    g = np.asarray(grad, np.float64)
    m1 = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v1 = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m1 / (1.0 - beta1 ** t)
    vh = v1 / (1.0 - beta2 ** t)
    p1 = p - lr * mh / (np.sqrt(vh) + eps)
    if frozen_rows is not None:
        fr = np.asarray(frozen_rows, bool)
        p1[fr] = p[fr]
        m1[fr] = np.asarray(m, np.float64)[fr]
        v1[fr] = np.asarray(v, np.float64)[fr]
    return p1, m1, v1


def compact(arr, keep):
    """Rows of arr whose keep flag is set, in their original order."""
    return np.asarray(arr)[np.asarray(keep, bool)]


ACT_W = (2.0, 0.1, 0.1)          # position, colour, scale weights (Sec. 3.2.2)


def activity_sample(d_means, d_sh, d_log_scales, weights=ACT_W) -> np.ndarray:
    """2 |d_mean| + 0.1 |d_sh| + 0.1 |d_log_scale| per Gaussian (row norms of one step's updates)."""
    n = np.asarray(d_means).shape[0]
    p = np.linalg.norm(np.asarray(d_means, np.float64).reshape(n, -1), axis=1)
    c = np.linalg.norm(np.asarray(d_sh, np.float64).reshape(n, -1), axis=1)
    s = np.linalg.norm(np.asarray(d_log_scales, np.float64).reshape(n, -1), axis=1)
    return weights[0] * p + weights[1] * c + weights[2] * s


def activity_prune(activity_sum, samples: int, threshold: float, trainable) -> np.ndarray:
    """keep = not (trainable and activity_sum / samples <= threshold)."""
    avg = np.asarray(activity_sum, np.float64) / samples
    return ~(np.asarray(trainable, bool) & (avg <= threshold))
