"""The learned warm start: the FP64 reference network is pinned by finite
differences; the GPU fp32 training gradient and the bf16 tensor-core inference
are checked against it; a warm-started run converges to the same state."""
import numpy as np
import pytest

from oracle import mlp as R
from paper_2203_06513_gb300 import inputs as I


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = R.init(1) + 0.05 * rng.normal(size=R.N_PARAMS)
    X = rng.normal(size=(7, 6))
    T = rng.normal(size=(7, 2))
    g = R.grad(theta, X, T)
    idx = rng.choice(R.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [0, 383, 384, 8768, 8896, 8897]])    # first/last of blocks
    h = 1e-6
    for i in idx:
        e = np.zeros(R.N_PARAMS)
        e[i] = h
        fd = (R.loss(theta + e, X, T) - R.loss(theta - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_reference_packing_and_relu():
    assert R.N_PARAMS == 8898
    z = np.array([-4.0, -1e-3, 0.0, 1e-3, 2.5])
    np.testing.assert_array_equal(R.relu(z), [0.0, 0.0, 0.0, 1e-3, 2.5])
    np.testing.assert_array_equal(R.relu_grad(z), [0.0, 0.0, 0.0, 1.0, 1.0])
    # away from the kink the derivative is the difference quotient
    zz = np.linspace(-4, 4, 100) + 0.0101
    h = 1e-6
    np.testing.assert_allclose(R.relu_grad(zz), (R.relu(zz + h) - R.relu(zz - h)) / (2 * h), atol=1e-8)


def _norm():
    return np.array([0.5, 0, 0, 0, 0, 0.05, 4.0, 5.0, 10.0, 3.0, 3.0, 10.0, 1.0, 1.0], dtype=np.float32)


def _normalise(X, norm):
    return (X - norm[:6]) * norm[6:12]


@pytest.mark.gpu
def test_gpu_gradient_matches_reference():
    torch = pytest.importorskip("torch")
    from paper_2203_06513_gb300 import pic
    rng = np.random.default_rng(3)
    theta = (R.init(2) + 0.05 * rng.normal(size=R.N_PARAMS)).astype(np.float32)
    norm = _norm()
    B = 1000          # 31 full 32-sample blocks and a ragged one
    X = np.column_stack([rng.random(B), rng.normal(0, 0.2, B), rng.normal(0, 0.05, B),
                         rng.normal(0, 0.2, B), rng.normal(0, 0.2, B), np.full(B, 0.05)]).astype(np.float32)
    T = rng.normal(size=(B, 2)).astype(np.float32)
    m = pic.Mlp(norm, theta)
    g = torch.zeros(R.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), g)
    Xn = _normalise(X.astype(np.float64), norm.astype(np.float64))
    Tn = T.astype(np.float64) / norm[12:14].astype(np.float64)
    ref_loss = R.loss(theta.astype(np.float64), Xn, Tn)
    ref = R.grad(theta.astype(np.float64), Xn, Tn)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    gg = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gg - ref)) <= 1e-4 * np.max(np.abs(ref))


@pytest.mark.gpu
def test_gpu_tensor_core_inference_matches_reference():
    torch = pytest.importorskip("torch")
    from paper_2203_06513_gb300 import pic
    rng = np.random.default_rng(4)
    theta = (R.init(5) + 0.05 * rng.normal(size=R.N_PARAMS)).astype(np.float32)
    norm = _norm()
    B = 4133          # not a multiple of the 32-marker warp tile
    X = np.column_stack([rng.random(B), rng.normal(0, 0.2, B), rng.normal(0, 0.05, B),
                         rng.normal(0, 0.2, B), rng.normal(0, 0.2, B), np.full(B, 0.05)]).astype(np.float32)
    m = pic.Mlp(norm, theta)
    Y = torch.zeros((B, 2), dtype=torch.float32, device="cuda")
    m.infer(torch.from_numpy(X).cuda(), Y)
    ref, _ = R.forward(theta.astype(np.float64), _normalise(X.astype(np.float64), norm.astype(np.float64)))
    ref = ref * norm[12:14]
    y = Y.cpu().numpy()
    # bf16 operands (8-bit mantissa) through four layers: a few 1e-3 of the output scale
    scale = np.max(np.abs(ref))
    print(f"\nbf16 tensor-core inference: max error {np.max(np.abs(y - ref)) / scale:.3e} of the output scale")
    assert np.max(np.abs(y - ref)) <= 2e-2 * scale      # measured 6.3e-3
    assert np.corrcoef(y[:, 0], ref[:, 0])[0, 1] > 0.999


@pytest.mark.gpu
def test_training_reduces_loss():
    torch = pytest.importorskip("torch")
    from paper_2203_06513_gb300 import pic
    rng = np.random.default_rng(6)
    B = 2048
    X = np.column_stack([rng.random(B), rng.normal(0, 0.2, B), rng.normal(0, 0.05, B),
                         rng.normal(0, 0.2, B), rng.normal(0, 0.2, B), np.full(B, 0.05)]).astype(np.float32)
    T = np.column_stack([np.sin(3 * X[:, 1]) + X[:, 2] * 4, X[:, 3] * X[:, 4] * 10]).astype(np.float32)
    m = pic.Mlp(_norm(), R.init(7).astype(np.float32))
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    l0 = m.grad(Xd, Td)
    for _ in range(300):
        m.train_step(Xd, Td, 3e-3)
    l1 = m.grad(Xd, Td)
    assert l1 < 0.1 * l0


@pytest.mark.gpu
def test_warm_started_run_reaches_the_same_fixed_point():
    """The Picard iteration runs to the same tolerance from the network's
    proposal: the state after two steps matches the oracle's (FP64 form)."""
    pytest.importorskip("torch")
    from oracle import oracle as O
    from paper_2203_06513_gb300 import pic
    w = I.Workload("wm", nx=32, degree=3, np=4096, seed=9, vth=0.2, pump=0.2)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, w.tol)
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    for _ in range(2):
        s = orc.step(s)
    m = pic.Mlp(_norm(), (0.3 * R.init(11)).astype(np.float32))
    g = pic.Pic(pic.Config.from_workload(w, warm_start=pic.PIC_WARM_MLP), x, p, ay, az, ey, ez)
    m.attach(g)
    g.step(2)
    st = g.state_numpy()
    d = np.mod(st["x"] - s.x + 0.5 * w.L, w.L) - 0.5 * w.L
    assert np.max(np.abs(d)) < 1e-12 * w.L
    assert np.max(np.abs(st["p"] - s.p)) < 1e-11
    assert np.max(np.abs(st["ex"] - s.ex)) < 1e-11
