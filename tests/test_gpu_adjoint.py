"""GPU parity of the differentiable leapfrog (FP32 forward, hand-written
adjoint, checkpointed reverse pass, torch.autograd) against the FP64
oracle's exact discrete adjoint.  Bar: relative L2 <= 1e-3 for each of
dL/dx0, dL/dv0, dL/dm (FP32 arithmetic against FP64)."""
import numpy as np
import pytest

from paper_0909_0879_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_0879_gb300 import _lib

    _lib.load()
    return torch


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_acc_and_vjp_kernels_match_oracle(torch_cuda, oracle_mod):
    torch = torch_cuda
    from paper_0909_0879_gb300 import _lib

    for n, eps in ((1, 1e-3), (37, 1e-3), (257, 0.0), (3000, 1e-3)):
        m, x, v = ics.plummer(n, 900 + n) if n > 1 else (np.ones(1), np.zeros((1, 3)), np.zeros((1, 3)))
        g = np.random.default_rng(n).normal(size=(n, 3))
        dx = torch.tensor(x, dtype=torch.float32, device="cuda")
        dm = torch.tensor(m, dtype=torch.float32, device="cuda")
        dg = torch.tensor(g, dtype=torch.float32, device="cuda")
        acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        gx = torch.empty_like(acc)
        gm = torch.empty(n, dtype=torch.float32, device="cuda")
        _lib.lf_acc(n, dx, dm, acc, eps=eps)
        _lib.lf_acc_vjp(n, dx, dm, dg, gx, gm, eps=eps)
        torch.cuda.synchronize()
        # the oracle sees the same float32-rounded inputs
        xr = dx.double().cpu().numpy()
        mr = dm.double().cpu().numpy()
        gr = dg.double().cpu().numpy()
        ra = oracle_mod.acc(mr, xr, eps)
        rgx, rgm = oracle_mod.acc_vjp(mr, xr, gr, eps)
        if n == 1:
            assert np.all(acc.cpu().numpy() == 0) and np.all(gm.cpu().numpy() == 0)
            continue
        assert rel_l2(acc.double().cpu().numpy(), ra) < 1e-5
        assert rel_l2(gx.double().cpu().numpy(), rgx) < 1e-4
        assert rel_l2(gm.double().cpu().numpy(), rgm) < 1e-4


@pytest.mark.parametrize("n", [65536, 131101, 262401])
@pytest.mark.parametrize("eps", [1e-3, 0.0])
def test_wide_acc_shape_large_n(torch_cuda, oracle_mod, eps, n):
    """N >= 65,536 takes the wide acceleration shape (4 particles per
    thread, packed pairs, 4 or 8 threads per particle group): the smallest
    such N, and two ragged ones, n = 131,101 (8 threads per group on 152
    SMs) and 262,401 (4 threads), against the FP64 oracle on 512 sampled
    particles, same float32-rounded inputs."""
    torch = torch_cuda
    from paper_0909_0879_gb300 import _lib

    m, x, v = ics.plummer(n, 905)
    dx = torch.tensor(x, dtype=torch.float32, device="cuda")
    dm = torch.tensor(m, dtype=torch.float32, device="cuda")
    acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    _lib.lf_acc(n, dx, dm, acc, eps=eps)
    torch.cuda.synchronize()
    xr = dx.double().cpu().numpy()
    mr = dm.double().cpu().numpy()
    sample = np.sort(np.random.default_rng(6).choice(n, 512, replace=False)).astype(np.int32)
    ra, _ = oracle_mod.force_jerk(mr, xr, np.zeros_like(xr), eps, idx=sample)
    got = acc.double().cpu().numpy()[sample]
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ra) < 1e-5


def test_leapfrog_adjoint_n4096(torch_cuda, oracle_mod):
    """N = 4096 Plummer, eps = 1e-3, 64 KDK steps of dt = 1/128 in FP32,
    checkpoints every 8 steps; L = sum |x(T) - y|^2 with y = x0 + N(0,0.05^2)
    (seed 5).  (a) The GPU gradient against the oracle's FP64 reverse sweep
    along the GPU's own FP32 trajectory: relative L2 <= 1e-4 (adjoint
    arithmetic).  (b) Against the oracle's fully FP64 run: relative L2 <=
    1e-2; the FP32 and FP64 trajectories separate through close encounters
    over the 64 steps, which bounds this agreement (about 4e-3 measured)."""
    torch = torch_cuda
    from paper_0909_0879_gb300 import _lib
    from paper_0909_0879_gb300.autograd import leapfrog

    n, eps, dt, steps = 4096, 1e-3, 1.0 / 128, 64
    m, x, v = ics.plummer(n, 1005)
    y = x + np.random.default_rng(5).normal(0.0, 0.05, x.shape)
    x0 = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    v0 = torch.tensor(v, dtype=torch.float32, device="cuda", requires_grad=True)
    mm = torch.tensor(m, dtype=torch.float32, device="cuda", requires_grad=True)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    xT, vT = leapfrog(x0, v0, mm, steps, dt, eps, ckpt_every=8)
    loss = ((xT - yt) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    g_gpu = [t.grad.double().cpu().numpy() for t in (x0, v0, mm)]
    # the GPU's own trajectory, every step (checkpoint interval 1)
    xw = x0.detach().clone()
    vw = v0.detach().clone()
    acc = torch.empty_like(xw)
    ck = torch.empty(_lib.lf_ckpt_floats(n, steps, 1), dtype=torch.float32, device="cuda")
    _lib.lf_forward(n, mm.detach(), xw, vw, acc, steps, dt, ck, eps=eps, ckpt_every=1)
    torch.cuda.synchronize()
    path = ck.view(steps, 2, n, 3)[:, 0].double().cpu().numpy()
    xs = np.concatenate([path, xw.double().cpu().numpy()[None]], axis=0)
    assert np.array_equal(xs[-1], xT.detach().double().cpu().numpy())
    mr = mm.detach().double().cpu().numpy()
    lx_T = 2.0 * (xs[-1] - yt.double().cpu().numpy())
    g_path = oracle_mod.leapfrog_adjoint_path(mr, xs, lx_T, np.zeros((n, 3)), eps, dt)
    e_path = [rel_l2(a, b) for a, b in zip(g_gpu, g_path)]
    xr = x0.detach().double().cpu().numpy()
    vr = v0.detach().double().cpu().numpy()
    L, gx, gv, gm = oracle_mod.leapfrog_loss_grad(mr, xr, vr, y, eps, dt, steps)
    e_full = [rel_l2(a, b) for a, b in zip(g_gpu, (gx, gv, gm))]
    print("loss gpu %.8e oracle %.8e; same-path rel L2 %s; FP64-run rel L2 %s"
          % (loss.item(), L, ["%.2e" % e for e in e_path], ["%.2e" % e for e in e_full]))
    assert abs(loss.item() - L) <= 1e-4 * L
    assert max(e_path) <= 1e-4
    assert max(e_full) <= 1e-2


def test_checkpoint_interval_does_not_change_gradients(torch_cuda):
    """Recomputing from checkpoints reproduces the forward pass exactly, so
    the gradient is bit-identical for any checkpoint interval."""
    torch = torch_cuda
    from paper_0909_0879_gb300.autograd import leapfrog

    n = 500
    m, x, v = ics.plummer(n, 3)
    grads = []
    for ck in (1, 3, 8, 64):
        x0 = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
        v0 = torch.tensor(v, dtype=torch.float32, device="cuda", requires_grad=True)
        mm = torch.tensor(m, dtype=torch.float32, device="cuda", requires_grad=True)
        xT, vT = leapfrog(x0, v0, mm, 20, 1.0 / 128, 1e-3, ckpt_every=ck)
        (xT.square().sum() + 0.5 * vT.square().sum()).backward()
        grads.append([t.grad.cpu().numpy() for t in (x0, v0, mm)])
    for g in grads[1:]:
        for a, b in zip(g, grads[0]):
            assert np.array_equal(a, b)
