"""Pins for the network oracle (oracle/conv3d.py): a single-tap kernel is a
plain shift, the convolution matches scipy's correlation, and the backward
pass matches central finite differences of the loss."""
import numpy as np
import pytest

from oracle import conv3d


def small_net(rng, ch=(2, 3, 3, 1)):
    Ws = [0.3 * rng.standard_normal((ch[l + 1], ch[l], 27)) for l in range(len(ch) - 1)]
    bs = [0.1 * rng.standard_normal(ch[l + 1]) for l in range(len(ch) - 1)]
    return Ws, bs


def test_single_tap_is_shift():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 1, 4, 5, 6))
    for t, (dz, dy, dx) in enumerate(conv3d.TAPS):
        W = np.zeros((1, 1, 27))
        W[0, 0, t] = 1.0
        z = conv3d.conv(x, W, np.zeros(1))
        ref = np.zeros_like(x)
        for k in range(4):
            for j in range(5):
                for i in range(6):
                    kk, jj, ii = k + dz, j + dy, i + dx
                    if 0 <= kk < 4 and 0 <= jj < 5 and 0 <= ii < 6:
                        ref[0, 0, k, j, i] = x[0, 0, kk, jj, ii]
        assert np.array_equal(z, ref)


def test_conv_matches_scipy_correlate():
    sc = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 2, 5, 4, 6))
    W = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    z = conv3d.conv(x, W, b)
    for co in range(3):
        ref = np.full(x.shape[2:], b[co])
        for ci in range(2):
            k = W[co, ci].reshape(3, 3, 3)
            ref += sc.correlate(x[0, ci], k, mode="constant", cval=0.0)
        assert np.allclose(z[0, co], ref, atol=1e-12)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    Ws, bs = small_net(rng)
    x = rng.standard_normal((2, 2, 4, 3, 5))
    t = rng.standard_normal((2, 1, 4, 3, 5))
    mask = (rng.random((4, 3, 5)) > 0.3).astype(float)

    def L(Ws_, bs_):
        acts = conv3d.forward(x, Ws_, bs_)
        return conv3d.loss_and_grad_out(acts[-1], t, mask)[0]

    acts = conv3d.forward(x, Ws, bs)
    _, g = conv3d.loss_and_grad_out(acts[-1], t, mask)
    dWs, dbs = conv3d.backward(acts, Ws, g)
    h = 1e-6
    for l in range(len(Ws)):
        for idx in [(0, 0, 0), (1, 1, 13), (0, 1, 26)]:
            idx = tuple(min(i, s - 1) for i, s in zip(idx, Ws[l].shape))
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            fd = (L(Wp, bs) - L(Wm, bs)) / (2 * h)
            assert abs(fd - dWs[l][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, dWs[l][idx])
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][0] += h
        bm[l][0] -= h
        fd = (L(Ws, bp) - L(Ws, bm)) / (2 * h)
        assert abs(fd - dbs[l][0]) <= 1e-6 * max(1.0, abs(fd))
