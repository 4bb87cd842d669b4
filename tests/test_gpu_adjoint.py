"""Adjoint of the collide-stream step: gradients of the time-averaged drag
J = (1/T) sum_t sum_p F_{p,x}(t) with respect to the particle positions and the body force,
against central finite differences of the FP64 oracle (the oracle's gradient) and of the
GPU forward itself, through the C ABI and the torch.autograd wrapper."""
import numpy as np
import pytest

import oracle as O
from parity_utils import oracle_params, perturbed_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1901_09745_gb300 import build
    build.build()
    import paper_1901_09745_gb300 as P
    P.lib()
    return P


def _case(lattice):
    if lattice == 19:
        X = np.array([[8.3, 9.1, 10.2], [15.6, 11.4, 9.3], [16.8, 3.3, 15.1]])
        return dict(lattice=19, n=(24, 22, 20), bc=(0, 0, 0), tau=0.7, body_force=(2e-5, -1e-5, 5e-6),
                    X=X, U=np.zeros((3, 3)), Om=np.zeros((3, 3)), r=np.array([4.1, 3.6, 3.3]))
    X = np.array([[12.3, 17.2, 0.0], [21.1, 19.9, 0.0], [33.5, 9.25, 0.0]])
    return dict(lattice=9, n=(44, 34, 1), bc=(0, 1, 0), tau=0.8, body_force=(3e-5, 1e-5, 0.0),
                X=X, U=np.zeros((3, 3)), Om=np.zeros((3, 3)), r=np.array([5.1, 3.9, 4.4]))


def _gpu_adjoint(P, case, f0, T, K, storage="f64", cap=0):
    ctx = P.lbm_create(case["lattice"], *case["n"], bc=case["bc"], tau=case["tau"],
                       body_force=case["body_force"], storage=storage, tile_cap=cap)
    P.lbm_set_populations(ctx, f0)
    P.lbm_set_particles(ctx, case["X"], case["U"], case["Om"], case["r"])
    out = P.lbm_adjoint_drag(ctx, T, K)
    P.lbm_destroy(ctx)
    return out


def _oracle_fd(case, f0, T, h):
    """Central differences of the oracle's J in every position coordinate (at h and 2h,
    Richardson-extrapolated; the h/2h disagreement flags a stencil that crosses a clamp kink
    of the solid fraction) and in every body-force component (J is smooth in F)."""
    dim = 2 if case["lattice"] == 9 else 3

    def J(X, F):
        c = dict(case, X=X, body_force=F)
        return O.drag(oracle_params(c), f0, T, X, case["r"])

    X0, F0 = case["X"], np.array(case["body_force"], dtype=float)
    gX = np.zeros_like(X0); gX2 = np.zeros_like(X0)
    for i in range(X0.shape[0]):
        for a in range(dim):
            for hh, out in ((h, gX), (2 * h, gX2)):
                Xp, Xm = X0.copy(), X0.copy()
                Xp[i, a] += hh; Xm[i, a] -= hh
                out[i, a] = (J(Xp, F0) - J(Xm, F0)) / (2 * hh)
    gF = np.zeros(3)
    for a in range(dim):
        hF = 1e-7
        Fp, Fm = F0.copy(), F0.copy()
        Fp[a] += hF; Fm[a] -= hF
        gF[a] = (J(X0, Fp) - J(X0, Fm)) / (2 * hF)
    return J(X0, F0), (4 * gX - gX2) / 3, np.abs(gX - gX2), gF


@pytest.mark.parametrize("lattice", [9, 19])
def test_adjoint_matches_oracle_finite_differences(P, lattice):
    case = _case(lattice)
    f0 = perturbed_state(case, 31, amp=2e-3)
    T, K = 12, 5
    J, dX, dF = _gpu_adjoint(P, case, f0, T, K, storage="f64")
    Jo, gX, kink, gF = _oracle_fd(case, f0, T, 5e-5)
    assert J == pytest.approx(Jo, rel=1e-11, abs=1e-16)
    scale = np.max(np.abs(gX))
    # smooth coordinates: the h/2h truncation gap is ~1e-6 of scale; a kink inside the
    # stencil moves one cell's share (about 1e-3 of scale or more)
    dim = 2 if lattice == 9 else 3
    smooth = (kink < 2e-5 * scale)[:, :dim]
    assert smooth.sum() >= 2 * dim
    assert np.max(np.abs(dX - gX)[:, :dim][smooth]) < 1e-6 * scale, (dX, gX)
    assert np.all(dX[:, dim:] == 0.0)
    assert np.allclose(dF, gF, rtol=1e-5, atol=1e-9 * np.max(np.abs(gF))), (dF, gF)


@pytest.mark.parametrize("lattice", [9, 19])
def test_adjoint_fp32_close_to_fp64(P, lattice):
    case = _case(lattice)
    f0 = perturbed_state(case, 32, amp=2e-3)
    J64, dX64, dF64 = _gpu_adjoint(P, case, f0, 12, 4, storage="f64")
    J32, dX32, dF32 = _gpu_adjoint(P, case, f0, 12, 4, storage="f32")
    assert J32 == pytest.approx(J64, rel=1e-4)
    assert np.max(np.abs(dX32 - dX64)) < 1e-3 * np.max(np.abs(dX64))
    assert np.max(np.abs(dF32 - dF64)) < 1e-3 * np.max(np.abs(dF64))


def test_checkpoint_interval_does_not_change_the_gradient(P):
    case = _case(19)
    f0 = perturbed_state(case, 33, amp=2e-3)
    ref = _gpu_adjoint(P, case, f0, 12, 12)
    for K in (1, 5, 7):
        J, dX, dF = _gpu_adjoint(P, case, f0, 12, K)
        # the forward state is re-run exactly; J sums forces through FP64 atomics whose
        # order varies between launches, so it agrees to FP64 rounding
        assert J == pytest.approx(ref[0], rel=1e-14, abs=0)
        assert np.allclose(dX, ref[1], rtol=1e-13, atol=1e-18)
        assert np.allclose(dF, ref[2], rtol=1e-13, atol=1e-18)


def test_autograd_function_backward(P):
    torch = pytest.importorskip("torch")
    case = _case(19)
    f0 = perturbed_state(case, 34, amp=2e-3)
    ctx = P.lbm_create(19, *case["n"], tau=case["tau"], body_force=case["body_force"], storage="f64")
    X = torch.tensor(case["X"], dtype=torch.float64, requires_grad=True)
    F = torch.tensor(case["body_force"], dtype=torch.float64, requires_grad=True)
    J = P.psc_drag(ctx, f0, X, case["r"], F, 10, 3)
    (2.0 * J).backward()
    Jr, dX, dF = _gpu_adjoint(P, case, f0, 10, 3)
    assert float(J.detach()) == pytest.approx(Jr, rel=1e-14)
    assert np.allclose(X.grad.numpy(), 2.0 * dX, rtol=1e-12, atol=0)
    assert np.allclose(F.grad.numpy(), 2.0 * dF, rtol=1e-12, atol=0)


def test_forward_and_backward_halves(P):
    """lbm_adjoint_forward + lbm_adjoint_backward give lbm_adjoint_drag's J and gradient;
    the backward can run twice; a later forward or a change of the particles or the body
    force makes the old token's backward fail instead of returning a stale gradient."""
    case = _case(19)
    f0 = perturbed_state(case, 35, amp=2e-3)
    Jr, dXr, dFr = _gpu_adjoint(P, case, f0, 9, 4)
    ctx = P.lbm_create(case["lattice"], *case["n"], bc=case["bc"], tau=case["tau"], body_force=case["body_force"],
                       storage="f64")
    P.lbm_set_populations(ctx, f0)
    P.lbm_set_particles(ctx, case["X"], case["U"], case["Om"], case["r"])
    J, tok = P.lbm_adjoint_forward(ctx, 9, 4)
    assert J == pytest.approx(Jr, rel=1e-14)
    assert P.lbm_get_info(ctx)["steps"] == 9
    for _ in range(2):
        dX, dF = P.lbm_adjoint_backward(ctx, tok)
        assert np.allclose(dX, dXr, rtol=1e-13, atol=1e-18)
        assert np.allclose(dF, dFr, rtol=1e-13, atol=1e-18)
    P.lbm_step(ctx, 2)                       # stepping on does not touch the checkpoints
    dX, _ = P.lbm_adjoint_backward(ctx, tok)
    assert np.allclose(dX, dXr, rtol=1e-13, atol=1e-18)
    _, tok2 = P.lbm_adjoint_forward(ctx, 3, 2)
    with pytest.raises(P.LbmError):
        P.lbm_adjoint_backward(ctx, tok)
    P.lbm_set_body_force(ctx, case["body_force"])
    with pytest.raises(P.LbmError):
        P.lbm_adjoint_backward(ctx, tok2)
    P.lbm_destroy(ctx)


def test_c4_adjoint_against_gpu_finite_differences():
    """The adjoint workload: D3Q19 128^3 periodic, tau 0.7, 200 static spheres r = 5, 500
    steps, checkpoint every 50, body force 1e-6; central differences (h = 1e-3 lu) of the GPU
    forward (FP64 storage, so the difference quotient is not swamped by FP32 rounding) on 8
    seeded particles, against the FP32 adjoint."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1901_09745_gb300 as P
    import synth
    w = synth.workload("c4")
    T, K, h = w["steps"], w["checkpoint"], 1e-3

    def drag(X, storage):
        # forward only: J from the forces of every step
        ctx = P.lbm_create(19, *w["n"], tau=w["tau"], body_force=w["body_force"], storage=storage)
        P.lbm_set_particles(ctx, X, w["U"], w["Om"], w["r"])
        J = 0.0
        for _ in range(T):
            P.lbm_step(ctx, 1)
            F, _T = P.lbm_get_forces(ctx)
            J += F[:, 0].sum() / T
        P.lbm_destroy(ctx)
        return J

    ctx = P.lbm_create(19, *w["n"], tau=w["tau"], body_force=w["body_force"], storage="f32")
    P.lbm_set_particles(ctx, w["X"], w["U"], w["Om"], w["r"])
    J, dX, dF = P.lbm_adjoint_drag(ctx, T, K)
    P.lbm_destroy(ctx)
    rng = np.random.default_rng(3001)
    pick = rng.choice(len(w["r"]), 8, replace=False)
    fd = np.zeros((8, 3))
    for k, i in enumerate(pick):
        for a in range(3):
            Xp, Xm = w["X"].copy(), w["X"].copy()
            Xp[i, a] += h; Xm[i, a] -= h
            fd[k, a] = (drag(Xp, "f64") - drag(Xm, "f64")) / (2 * h)
    scale = np.max(np.abs(fd))
    err = np.abs(dX[pick] - fd)
    # at most two of the 24 coordinates may sit on a clamp kink within +-h
    assert np.sum(err > 2e-2 * scale) <= 2, (err / scale)
