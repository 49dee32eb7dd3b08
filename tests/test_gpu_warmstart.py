"""GPU warm start: the BF16 network kernels against the FP64 network oracle, and a small training
run whose predicted starting points reduce the SGP iterations to the same discrepancy stop."""
import numpy as np
import pytest

from oracle import warmstart_oracle as WO
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu


def _bf16_round(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def test_network_forward_and_gradients_match_oracle(gpu):
    import torch
    from paper_1210_2258_b300 import warmstart as W
    rng = np.random.default_rng(2)
    p = {"w1": rng.standard_normal((32, 9)) * 0.3, "b1": rng.standard_normal(32) * 0.1,
         "w6": rng.standard_normal((9, 32)) * 0.1, "b6": rng.standard_normal(1) * 0.1}
    for i in range(2, 6):
        p[f"w{i}"] = _bf16_round(rng.standard_normal((32, 9, 32)) * 0.1)
        p[f"b{i}"] = rng.standard_normal(32) * 0.1
    B, H, Wd = 2, 32, 32
    x0 = rng.standard_normal((B, H, Wd)).astype(np.float32)
    t = rng.standard_normal((B, H, Wd)).astype(np.float32)
    net = W.WarmStartNet(seed=0)
    net.set_params(p)
    bf = net.buffers(B, H, Wd)
    bf["x0"].copy_(torch.from_numpy(x0))
    bf["tgt"].copy_(torch.from_numpy(t))
    net.loss_and_grad(bf, B, H, Wd)
    torch.cuda.synchronize()
    ref = WO.Net(p)
    loss, g = ref.loss_and_grads(x0.astype(np.float64), t.astype(np.float64))
    z = bf["z"].double().cpu().numpy()
    assert rel_l2(z, ref.cache["z"]) <= 2e-2
    assert abs(float(bf["loss"].item()) - loss) <= 3e-2 * loss
    gp = net.g.cpu().numpy()
    for name, (a, n) in net.off.items():
        gg = gp[a:a + n]
        rr = g[name].reshape(-1)
        assert rel_l2(gg, rr) <= 5e-2, (name, rel_l2(gg, rr))


def test_trained_warm_start_reduces_iterations(gpu):
    from paper_1210_2258_b300 import warmstart as W
    train_scs = W.make_scenes(192, 128, seed=10)
    g, f, b, its = W.sgp_solutions(train_scs, max_iter=400)
    net = W.WarmStartNet(seed=1)
    losses = W.train(net, g, f, b, epochs=4, batch=16, lr=3e-3)
    assert losses[-1] < losses[0]
    ev = W.evaluate(net, W.make_scenes(24, 128, seed=99), max_iter=2000, batch=24)
    done = (ev["flat_iters"] < 2000) & (ev["warm_iters"] < 2000)
    assert done.sum() >= 12
    assert ev["warm_iters"][done].mean() < ev["flat_iters"][done].mean()


def test_adam_kernel_matches_oracle(gpu):
    """ws_adam (FP32) against the FP64 Adam of the oracle over four steps of varied gradients."""
    import torch
    from paper_1210_2258_b300 import warmstart as W
    rng = np.random.default_rng(5)
    n = 9000
    p0 = rng.standard_normal(n).astype(np.float32)
    gs = [(rng.standard_normal(n) * 10.0 ** rng.uniform(-4, 1, n)).astype(np.float32) for _ in range(4)]
    p = torch.from_numpy(p0.copy()).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    L = W._lib()
    for t, g in enumerate(gs, start=1):
        gd = torch.from_numpy(g).cuda()
        assert L.ws_adam(p.data_ptr(), m.data_ptr(), v.data_ptr(), gd.data_ptr(), n, 1e-3, 0.9, 0.999, 1e-8, t,
                         torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    # the kernel receives lr, beta1, beta2 and eps as float32: the oracle runs with those values
    f32 = lambda x: float(np.float32(x))
    rp, rm, rv = WO.adam(p0.astype(np.float64), [g.astype(np.float64) for g in gs], f32(1e-3), b1=f32(0.9),
                         b2=f32(0.999), eps=f32(1e-8))
    assert np.max(np.abs(p.double().cpu().numpy() - rp)) <= 1e-6 * np.max(np.abs(rp)) + 1e-7
    assert rel_l2(m.double().cpu().numpy(), rm) <= 1e-6
    assert rel_l2(v.double().cpu().numpy(), rv) <= 1e-6
