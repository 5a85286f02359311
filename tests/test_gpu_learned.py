"""Learned preconditioner: the network kernels against the float64 oracle
(oracle/conv3d.py), training on the GPU, and the gain over Jacobi-PCG.

Stated error: the GPU network stores weights and activations in BF16 and
accumulates in float32, so against the float64 oracle (fed the same
BF16-rounded weights and inputs) the output agrees to 3e-2 and the parameter
gradients to 5e-2 (relative, Frobenius) on a 4 x 5 x 6 box."""
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


def test_untrained_network_is_jacobi(env):
    """The last layer starts at zero, so the flexible CG with the untrained net
    takes the same iterations as Jacobi-PCG and gives the same solution."""
    torch, cr = env
    from paper_1808_05510_gb300 import learned

    p = synth.toy2d()
    net = cr.ConvNet(learned.box_mask(p.grid_y).shape, batch_cap=1)
    res = learned.compare_iterations(p, net, [2])
    for r in res:
        assert r["rel_diff"] < 1e-6
        assert abs(r["iters_learned"] - r["iters_jacobi"]) <= 2
    net.close()


def test_learned_preconditioner_gain(env):
    """Trained on the solver's own u-side systems of three toy problems, the
    network cuts flexible-CG iterations on a held-out problem, same solution."""
    torch, cr = env
    from paper_1808_05510_gb300 import learned

    train = [synth.toy2d(seed=s) for s in (11, 12, 13)]
    pairs = []
    for k, p in enumerate(train):
        pairs += learned.make_pairs(p, [0, 2, 4, 6, 8], n_random=6, seed=k)
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
