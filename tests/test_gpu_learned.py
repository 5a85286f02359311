"""Learned preconditioner: the network kernels against the float64 oracle
(oracle/conv3d.py), training on the GPU, and the gain over Jacobi-PCG.

Stated errors (relative, Frobenius, 4 x 5 x 6 box, 2 samples):
- the same kernel templates instantiated with float64 storage and
  accumulation (cr_net_check_f64): output, loss and gradients to 1e-10;
- the BF16 network (BF16 weights and activations, float32 accumulation)
  against the oracle run with the same BF16 storage (weights, input and every
  hidden activation rounded to BF16 as the kernels store them): 1e-2;
- the BF16 network against the exact float64 network (only weights and input
  rounded): 3e-2 for the output, 5e-2 for the gradients.  That gap is the BF16
  storage of the hidden activations (8 significant bits, about 4e-3 per value,
  compounded over four layers of 27 x 16 taps), not the kernels."""
import numpy as np
import pytest

from oracle import conv3d
from paper_1808_05510_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1808_05510_gb300 import build

    build.build()
    from paper_1808_05510_gb300 import conreg

    conreg.load()
    return torch, conreg


CH = [2, 16, 16, 16, 1]


def unpack(flat):
    Ws, bs, k = [], [], 0
    for l in range(4):
        n = CH[l + 1] * CH[l] * 27
        Ws.append(flat[k:k + n].reshape(CH[l + 1], CH[l], 27).astype(np.float64))
        k += n
        bs.append(flat[k:k + CH[l + 1]].astype(np.float64))
        k += CH[l + 1]
    return Ws, bs


def bf16(a, torch):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def test_network_forward_and_gradients_match_oracle(env):
    torch, cr = env
    dims = (4, 5, 6)
    net = cr.ConvNet(dims, batch_cap=2, seed=3)
    rng = np.random.default_rng(5)
    flat = (0.25 * rng.standard_normal(cr.ConvNet.param_count())).astype(np.float32)
    net.set_params(flat)
    x = rng.standard_normal((2, 2) + dims).astype(np.float32)
    t = rng.standard_normal((2,) + dims).astype(np.float32)
    mask = (rng.random(dims) > 0.25).astype(np.uint8)
    dev = torch.device("cuda")
    xd, td, md = torch.tensor(x, device=dev), torch.tensor(t, device=dev), torch.tensor(mask, device=dev)
    out = net.forward(xd).cpu().numpy().astype(np.float64)
    Ws, bs = unpack(flat)
    Ws = [bf16(w, torch) for w in Ws]
    acts = conv3d.forward(bf16(x, torch), Ws, bs)
    ref = acts[-1][:, 0]
    assert np.linalg.norm(out - ref) <= 3e-2 * np.linalg.norm(ref)
    loss, g = net.gradients(xd, td, md)
    loss_ref, gout = conv3d.loss_and_grad_out(acts[-1], t[:, None].astype(np.float64), mask.astype(np.float64))
    assert abs(loss - loss_ref) <= 3e-2 * loss_ref
    dWs, dbs = conv3d.backward(acts, Ws, gout)
    gW, gb = unpack(g)
    for l in range(4):
        assert np.linalg.norm(gW[l] - dWs[l]) <= 5e-2 * np.linalg.norm(dWs[l]), l
        assert np.linalg.norm(gb[l] - dbs[l]) <= 5e-2 * np.linalg.norm(dbs[l]) + 1e-7, l
    net.close()


def random_case(cr, seed, dims=(4, 5, 6), B=2):
    rng = np.random.default_rng(seed)
    flat = 0.25 * rng.standard_normal(cr.ConvNet.param_count())
    x = rng.standard_normal((B, 2) + dims)
    t = rng.standard_normal((B,) + dims)
    mask = (rng.random(dims) > 0.25).astype(np.uint8)
    return flat, x, t, mask


def oracle_all(x, Ws, bs, t, mask, round_fn=None):
    """Oracle forward, loss and gradients; round_fn (if given) is applied to the
    input and to every hidden activation, as the network's storage does."""
    r = round_fn or (lambda a: a)
    acts = [r(x)]
    for l in range(4):
        z = conv3d.conv(acts[-1], Ws[l], bs[l])
        acts.append(r(np.maximum(z, 0.0)) if l < 3 else z)
    loss, gout = conv3d.loss_and_grad_out(acts[-1], t[:, None], mask.astype(np.float64))
    dWs, dbs = conv3d.backward(acts, Ws, gout)
    return acts[-1][:, 0], loss, dWs, dbs


def test_float64_template_matches_oracle(env):
    """cr_net_check_f64 runs the network's own kernel templates in float64."""
    torch, cr = env
    flat, x, t, mask = random_case(cr, 8)
    out, loss, g = cr.ConvNet.check_f64((4, 5, 6), flat, x, t, mask)
    Ws, bs = unpack(flat)
    ref, loss_ref, dWs, dbs = oracle_all(x, Ws, bs, t, mask)
    assert np.linalg.norm(out - ref) <= 1e-10 * np.linalg.norm(ref)
    assert abs(loss - loss_ref) <= 1e-10 * loss_ref
    gW, gb = unpack(g)
    for l in range(4):
        assert np.linalg.norm(gW[l] - dWs[l]) <= 1e-10 * np.linalg.norm(dWs[l]), l
        assert np.linalg.norm(gb[l] - dbs[l]) <= 1e-10 * np.linalg.norm(dbs[l]), l


def test_bf16_network_matches_oracle_with_bf16_storage(env):
    torch, cr = env
    dims = (4, 5, 6)
    flat, x, t, mask = random_case(cr, 9)
    flat = flat.astype(np.float32)
    net = cr.ConvNet(dims, batch_cap=2, seed=3)
    net.set_params(flat)
    dev = torch.device("cuda")
    xd = torch.tensor(x.astype(np.float32), device=dev)
    td = torch.tensor(t.astype(np.float32), device=dev)
    md = torch.tensor(mask, device=dev)
    out = net.forward(xd).cpu().numpy().astype(np.float64)
    loss, g = net.gradients(xd, td, md)
    net.close()
    Ws, bs = unpack(flat)
    Ws = [bf16(w, torch) for w in Ws]
    r = lambda a: bf16(a, torch)  # noqa: E731
    ref, loss_ref, dWs, dbs = oracle_all(x.astype(np.float32).astype(np.float64), Ws, bs,
                                         t.astype(np.float32).astype(np.float64), mask, round_fn=r)
    assert np.linalg.norm(out - ref) <= 1e-2 * np.linalg.norm(ref)
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref
    gW, gb = unpack(g)
    for l in range(4):
        assert np.linalg.norm(gW[l] - dWs[l]) <= 1e-2 * np.linalg.norm(dWs[l]), l
        assert np.linalg.norm(gb[l] - dbs[l]) <= 1e-2 * np.linalg.norm(dbs[l]) + 1e-7, l


def test_untrained_network_is_jacobi(env):
    """The last layer starts at zero, so the flexible CG with the untrained net
    is Jacobi-PCG with the Polak-Ribiere beta: the same solution, and the same
    iterations up to rounding (the two betas agree only in exact arithmetic)."""
    torch, cr = env
    from paper_1808_05510_gb300 import learned

    p = synth.toy2d()
    net = cr.ConvNet(learned.box_mask(p.grid_y).shape, batch_cap=1)
    res = learned.compare_iterations(p, net, [2])
    for r in res:
        assert r["rel_diff"] < 1e-6
        assert abs(r["iters_learned"] - r["iters_jacobi"]) <= max(2, 0.05 * r["iters_jacobi"])
    net.close()


def test_learned_preconditioner_gain(env):
    """Trained on the solver's own u-side systems of three toy problems, the
    network cuts flexible-CG iterations on a held-out problem, same solution."""
    torch, cr = env
    from paper_1808_05510_gb300 import learned

    train = [synth.toy2d(seed=s) for s in (11, 12, 13)]
    pairs = []
    for k, p in enumerate(train):
        pairs += learned.make_pairs(p, [0, 2, 4, 6, 8], n_random=6, seed=k, sides=(0,))
    net = cr.ConvNet(learned.box_mask(train[0].grid_y).shape, batch_cap=8, seed=1)
    hist = learned.train(net, pairs, steps=400, lr=2e-3, batch=8)
    assert np.mean(hist[-20:]) < 0.8 * np.mean(hist[:20])
    test = synth.toy2d(seed=99)
    res = learned.compare_iterations(test, net, [0, 3, 6])
    print(res)
    for r in res:
        assert r["rel_diff"] < 1e-6
    assert sum(r["iters_learned"] for r in res) < sum(r["iters_jacobi"] for r in res)
    net.close()


def test_learned_preconditioner_both_sides_blob_mask(env):
    """Trained on both sides of 3-D blob-mask problems: the flexible CG reaches
    the Jacobi-PCG solution on held-out u- and v-side systems."""
    torch, cr = env
    from paper_1808_05510_gb300 import learned

    train = [synth.masked3d(seed=s) for s in (21, 22)]
    # the same box for every problem of the family
    net, hist, npairs = learned.train_for(train, [0, 3, 6], steps=200, n_random=2, batch=8)
    assert npairs > 20 and np.mean(hist[-20:]) < np.mean(hist[:20])
    test = synth.masked3d(seed=29)
    res = learned.compare_iterations(test, net, [0, 4], sides=(0, 1))
    print(res)
    for r in res:
        assert r["rel_diff"] < 1e-6
    net.close()


@pytest.mark.parametrize("judge,losses", [(0, 2), (1, 3)], ids=["by-time", "by-iterations"])
def test_garbage_network_falls_back_to_jacobi(env, judge, losses):
    """A network with large random weights: every learned solve stagnates, is
    finished by Jacobi-PCG (same solution), and after two (judged by time) or
    three (by iterations) fallbacks in a row the learned form is switched off
    for that side."""
    torch, cr = env
    from paper_1808_05510_gb300 import learned

    p = synth.toy2d()
    net = cr.ConvNet(learned.box_mask(p.grid_y).shape, batch_cap=1)
    rng = np.random.default_rng(5)
    net.set_params((5.0 * rng.standard_normal(net.param_count())).astype(np.float32))
    with cr.ConReg.from_problem(p, r_cap=4, pcg_tol=1e-9, pcg_maxit=100000) as gj, \
            cr.ConReg.from_problem(p, r_cap=4, pcg_tol=1e-9, pcg_maxit=100000,
                                   precond=cr.CR_PRECOND_LEARNED, learned_judge=judge) as gl:
        gl.cr_set_voxel_grid(0, p.grid_y.mask)
        gl.cr_set_voxel_grid(1, p.grid_x.mask)
        gl.cr_set_preconditioner(net)
        gl.cr_get_stats(reset=True)
        v = gj.cr_apply_residual(np.ones(p.ny), trans=True)
        v /= np.linalg.norm(v)
        r = gj.cr_apply_residual(v)
        ej, itj = gj.cr_solve_u(v, r)
        its = []
        for _ in range(5):
            el, itl = gl.cr_solve_u(v, r)
            its.append(itl)
            assert np.linalg.norm(el - ej) <= 1e-6 * np.linalg.norm(ej)
        st = gl.cr_get_stats()
        assert its[0] == itj  # the judge run is Jacobi-PCG
        assert st["learned_fallbacks"] == losses and st["learned_solves"] == 0
        assert st["learned_off"] & 1
        assert all(it == itj for it in its[losses + 1:])  # switched off: plain Jacobi-PCG again
    net.close()
