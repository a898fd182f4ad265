"""The forward-difference gradient on the GPU (lbm_set_gradient).  Section 4
of the paper first tried grad(rho) = rho(x+1) - rho(x) and found the model
unstable as c_e approaches 1, which led to the central difference.  The GPU
forward-difference step must equal the FP64 oracle's forward-difference step
(oracle.run(..., grad="forward")), and reproduce the instability: at c_e =
0.95 a plane wave grows at the rate of the linear analysis's largest
eigenvalue, while the central difference keeps it bounded."""
import numpy as np
import pytest

from oracle import linear, oracle
from paper_0707_2437_gb300 import workloads

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _gpu(lbm, nx, ny, tau, c2, fields, steps, grad):
    with lbm.Grid(nx, ny, tau, c2, "f32") as g:
        g.set_gradient(grad)
        assert g.get_gradient() == grad
        g.init(*fields)
        g.step(steps)
        return g.moments()


def _oracle(nx, ny, tau, c2, fields, steps, grad):
    f = oracle.init(*fields)
    oracle.run(f, tau, 1.0 / 3.0 - c2, steps, grad=grad)
    return oracle.moments(f)


@pytest.mark.parametrize("nx,ny", [(64, 16), (37, 23), (256, 9)])
def test_forward_difference_matches_oracle(lbm, nx, ny):
    """A stable setting (c_e = 0.5), 300 steps, amplitude 1e-3, odd sizes and
    several strips: within the FP32 bar of the other parity tests (1e-6)."""
    tau, c2, steps = 0.8, 0.25, 300
    fields = workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx + ny)
    got = _gpu(lbm, nx, ny, tau, c2, fields, steps, "forward")
    ref = _oracle(nx, ny, tau, c2, fields, steps, "forward")
    err = max(np.abs(a - b).max() for a, b in zip(got, ref))
    print(f"forward {nx}x{ny}: max |GPU - oracle| = {err:.3e}")
    assert err <= 1e-6
    # The two schemes differ by far more than the parity error.
    cen = _gpu(lbm, nx, ny, tau, c2, fields, steps, "central")
    assert np.abs(cen[0] - got[0]).max() > 100 * max(err, 1e-10)


def _dominant_mode(nx, tau, alpha, amp):
    """The fastest-growing forward-difference plane wave along x of an
    nx-periodic grid (linear analysis), as a perturbation df[i, x] of the
    rest state with density amplitude amp, and its |lambda|."""
    best = None
    for m in range(nx):
        k = 2 * np.pi * m / nx
        lam, vec = linear.eigen(k, 0.0, tau, alpha, "forward")
        j = int(np.argmax(np.abs(lam)))
        if best is None or abs(lam[j]) > best[0]:
            best = (abs(lam[j]), k, vec[:, j])
    lam, k, a = best
    a = a * (amp / abs(a.sum()))
    x = np.arange(nx)
    return (a[:, None] * np.exp(1j * k * x)[None, :]).real, lam


EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]


def _to_stored(h):
    """The stored form of pre-collision deviations h_i(x): the step pulls
    direction i from x - e_i, so the buffer holds h_i(x + e_i) at x."""
    return np.stack([np.roll(h[i], (-EY[i], -EX[i]), axis=(0, 1)) for i in range(9)])


def _drho_gpu(state, nx, ny):
    """Density deviation of the pre-collision distributions the next step
    pulls from a checkpoint."""
    h = np.frombuffer(state.tobytes(), dtype=np.float32).reshape(9, ny, nx).astype(np.float64)
    pre = np.stack([np.roll(h[i], (EY[i], EX[i]), axis=(0, 1)) for i in range(9)])
    return np.tensordot(W, pre, axes=1)


def test_forward_difference_unstable_where_central_is_stable(lbm):
    """c_e = 0.95, tau = 0.8, a 128 x 4 grid started in the fastest-growing
    forward-difference plane wave (density amplitude 1e-10, so the run stays
    linear).  Forward: after 300 steps the wave has grown by |lambda|^300
    (2e6) on the GPU, the same as in the oracle site by site.  Central, from
    the same state: it stays bounded."""
    nx, ny, tau, ce, steps = 128, 4, 0.8, 0.95, 300
    c2 = ce * ce
    alpha = 1.0 / 3.0 - c2
    df, lam = _dominant_mode(nx, tau, alpha, 1e-10)
    assert lam > 1.04
    f0 = W[:, None, None] + np.broadcast_to(df[:, None, :], (9, ny, nx))
    h0 = np.broadcast_to(df[:, None, :], (9, ny, nx)) / W[:, None, None]
    d0 = np.abs(np.tensordot(W, h0, axes=1)).max()
    s0 = np.ascontiguousarray(_to_stored(h0).astype(np.float32))
    out = {}
    for grad in ("forward", "central"):
        with lbm.Grid(nx, ny, tau, c2, "f32") as g:
            g.set_gradient(grad)
            g.set_state(s0.view(np.uint8).ravel(), 0)
            g.step(steps)
            out[grad] = _drho_gpu(g.get_state()[0], nx, ny)
    f = np.ascontiguousarray(f0)
    oracle.run(f, tau, alpha, steps, grad="forward")
    ref = f.sum(axis=0) - 1.0
    grow = np.abs(out["forward"]).max() / d0
    grow_ref = np.abs(ref).max() / d0
    print(f"forward growth over {steps} steps: GPU {grow:.5e}, oracle {grow_ref:.5e}, "
          f"|lambda|^n {lam ** steps:.5e}")
    assert abs(grow / lam ** steps - 1) < 1e-2
    assert abs(grow_ref / lam ** steps - 1) < 1e-2
    assert np.abs(out["forward"] - ref).max() <= 1e-3 * np.abs(ref).max()
    assert np.abs(out["central"]).max() <= 2 * d0


def test_forward_difference_argument_checks(lbm):
    with lbm.Grid(64, 8, 0.8, 0.2, "f16d") as g:
        with pytest.raises(Exception):
            g.set_gradient("forward")
    with lbm.Grid(64, 8, 0.8, 0.2, "f32") as g:
        g.set_c2_field(np.full((8, 64), 0.2))
        with pytest.raises(Exception):
            g.set_gradient("forward")
    with lbm.Grid(64, 8, 0.8, 0.2, "f32") as g:
        g.set_gradient("forward")
        with pytest.raises(Exception):
            g.set_c2_field(np.full((8, 64), 0.2))
        with pytest.raises(Exception):
            lbm.Batch([g])
        g.set_gradient("central")
        b = lbm.Batch([g])
        b.close()
