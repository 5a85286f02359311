"""The synthetic input recipe: the generators produce the shapes and structure
that the workloads claim (mask sizes and connectivity, Laplacian, injections,
observation mask, W_true, noise), checked against independent constructions
(brute-force pair loops, dense products, closed-form kernel values)."""
import math

import numpy as np
import pytest
from scipy import ndimage

from paper_1808_05510_gb300 import synth


def brute_laplacian(mask):
    """Deg - Adj of the face-adjacency graph, by a loop over voxel pairs."""
    coords = [tuple(c) for c in np.argwhere(mask)]
    n = len(coords)
    L = np.zeros((n, n))
    for i in range(n):
        for k in range(n):
            if i != k and sum(abs(a - b) for a, b in zip(coords[i], coords[k])) == 1:
                L[i, k] = -1.0
    L[np.diag_indices(n)] = -L.sum(axis=1)
    return L


@pytest.mark.parametrize("shape,seed", [((5, 6, 4), 0), ((7, 9), 1), ((11,), 2)])
def test_laplacian_matches_brute_force(shape, seed):
    rng = np.random.default_rng(seed)
    mask = rng.random(shape) < 0.6
    L = synth.grid_laplacian(synth.Grid(mask))
    assert np.array_equal(L.to_dense(), brute_laplacian(mask))
    for i in range(L.n):
        cols = L.col[L.rowptr[i]:L.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)  # ascending, no duplicates


@pytest.fixture(scope="module")
def visual():
    return synth.visual_cortex()


def test_visual_cortex_shape(visual):
    p = visual
    assert p.grid_x.mask.shape == (40, 40, 40)
    assert abs(p.nx - 7500) <= 0.05 * 7500 and p.nx == p.ny
    assert p.m == 28 and p.lam == 100.0
    _, ncomp = ndimage.label(p.grid_x.mask, structure=ndimage.generate_binary_structure(3, 1))
    assert ncomp == 1  # one face-connected component
    L = p.Lx.to_dense()
    deg = np.diag(L)
    assert deg.max() <= 6 and deg.min() >= 1
    assert np.allclose(L.sum(axis=1), 0.0) and np.array_equal(L, L.T)


def test_injections_and_observation_mask(visual):
    """X: Gaussian blobs of amplitude 1 and sigma 2 voxels centred on a mask voxel,
    zero beyond 3 sigma; Omega = 1{X <= 0.4}; Y vanishes where Omega does."""
    p = visual
    X = np.asarray(p.X.toarray() if hasattr(p.X, "toarray") else p.X)
    c = p.grid_x.coords().astype(np.float64)
    for a in range(p.m):
        col = X[:, a]
        i0 = int(np.argmax(col))
        assert col[i0] == 1.0
        d2 = ((c - c[i0]) ** 2).sum(1)
        nz = col != 0.0
        assert np.all(d2[nz] <= 36.0)
        assert np.allclose(col[nz], np.exp(-d2[nz] / 8.0), rtol=0, atol=1e-15)
    Om = np.asarray(p.Omega)
    assert np.array_equal(Om, (X <= 0.4).astype(np.uint8))
    assert np.all(np.asarray(p.Y)[Om == 0] == 0.0)


def test_w_true_kernel_values():
    """W_true(p_i, p_k) = exp(-|p_i - p_k|^2 / 0.4^2) + 0.9 exp(-(|p_k - a|^2 + |p_i - b|^2) / 0.2^2)
    with a = 0.8, b = 0.1 per axis: its special values."""
    a3, b3 = np.full((1, 3), 0.8), np.full((1, 3), 0.1)
    # source at a, target at b: the second bump is exactly 0.9; the first is exp(-3 * 0.49 / 0.16)
    w = synth.w_true_block(b3, a3)[0, 0]
    assert math.isclose(w, math.exp(-3 * 0.49 / 0.16) + 0.9, rel_tol=1e-15)
    # target at 1 (far from b), source at 0 (far from a): both terms in closed form
    w = synth.w_true_block(np.ones((1, 3)), np.zeros((1, 3)))[0, 0]
    assert math.isclose(w, math.exp(-3.0 / 0.16) + 0.9 * math.exp(-(3 * 0.64 + 3 * 0.81) / 0.04), rel_tol=1e-14)
    # the first term is symmetric, the second is not
    rng = np.random.default_rng(3)
    P = rng.random((6, 2))
    W = synth.w_true_block(P, P)
    bump = 0.9 * np.exp(-(((P - 0.8) ** 2).sum(1)[None, :] + ((P - 0.1) ** 2).sum(1)[:, None]) / 0.04)
    S = W - bump
    assert np.allclose(S, S.T, atol=1e-15) and np.allclose(np.diag(S), 1.0, atol=1e-15)


def test_tilewise_y_equals_dense_product():
    """make_Y applies W_true tile-wise over the support of X; without noise that is
    (W_true X) o Omega from the dense W_true."""
    p = synth.toy2d()
    X = np.asarray(p.X.toarray() if hasattr(p.X, "toarray") else p.X)
    Om = np.asarray(p.Omega)
    Y0 = synth.make_Y(p.grid_y, p.grid_x, X, Om, np.random.default_rng(0), 0.0, chunk=37)
    assert np.allclose(Y0, (p.W_true @ X) * Om, rtol=1e-13, atol=1e-13)
    # the noise is Gaussian at 1 % of the largest observed entry
    E = (np.asarray(p.Y) - (p.W_true @ X) * Om)[Om == 1]
    scale = 0.01 * np.abs((p.W_true @ X) * Om).max()
    assert abs(E.std() / scale - 1.0) < 0.1 and abs(E.mean()) < 0.1 * scale


def test_paper_toy_recipe():
    """Sec. 3.1: 200-point chain, 5 box injections of width 0.12 + 0.1 U(0, 1), Omega = 1 - X."""
    p = synth.paper_toy()
    X = np.asarray(p.X)
    assert p.nx == p.ny == 200 and p.m == 5
    assert set(np.unique(X)) <= {0.0, 1.0}
    assert np.array_equal(np.asarray(p.Omega), (1 - X).astype(np.uint8))
    x = p.grid_x.unit_coords()[:, 0]
    for a in range(5):
        inside = x[X[:, a] == 1.0]
        assert 0.12 - 2.0 / 199 <= inside.max() - inside.min() <= 0.22
        assert np.all(np.diff(np.flatnonzero(X[:, a])) == 1)  # one contiguous box
    L = p.Lx.to_dense()
    assert L[0, 0] == 1.0 and L[1, 1] == 2.0  # chain: end degree 1


def test_shell_mask_size():
    mask = synth.shell_mask((48, 32, 40), 6000)
    assert abs(int(mask.sum()) - 6000) <= 0.1 * 6000
