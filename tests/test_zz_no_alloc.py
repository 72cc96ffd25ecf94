"""The allocation-free fluid step against the regular entry points.

Some callers cannot allocate device memory, nor give the library a workspace
(their host framework owns every allocation); susp_fluid_step_noalloc serves
them with a static scratch array inside the library.  This test drives it
through the C ABI on two consecutive steps of a sheared, particle-free FP32
box and compares populations and viscous stress with susp_create /
susp_set_populations / susp_step / susp_stress, within the FP32 tolerance of
the other parity tests (2e-5 relative).  It lives in its own file, collected
last, and passes both alone and after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,tau,rate", [((37, 21, 13), 0.8, 3.7e-3), ((32, 16, 8), 1.0, 1e-3)])
def test_noalloc_step_matches_regular_step_twice(shape, tau, rate):
    import torch
    import oracle as O
    from paper_1904_02929_gb300 import inputs as I
    from paper_1904_02929_gb300 import susp as S

    nx, ny, nz = shape
    _, w, _ = O.lattice()
    f0 = I.random_populations(nx, ny, nz, seed=77, amplitude=0.03, weights=w).astype(np.float32)

    # regular path: workspace owned by the binding, two steps
    g = S.Suspension(nx, ny, nz, precision="fp32", tau=tau)
    g.set_populations(f0.astype(np.float64))
    sh = S.make_shear(kind=0, rate=rate)
    g.step(1, sh)
    f1_ref = g.populations()
    s1_ref, _ = g.stress(S.VISCOUS)
    g.step(1, sh)
    f2_ref = g.populations()
    s_avg, _ = g.stress(S.VISCOUS)
    s2_ref = 2.0 * s_avg - s1_ref

    # allocation-free path: the caller owns only inputs and outputs
    dev = torch.device("cuda")
    a = torch.from_numpy(f0.ravel()).to(dev)
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    visc = torch.empty(9, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    u_le = ny * rate
    S.susp_fluid_step_noalloc(nx, ny, nz, tau, 0.0, u_le, a.data_ptr(), b.data_ptr(),
                              visc.data_ptr(), stream)
    s1 = visc.cpu().numpy().reshape(3, 3).copy()
    delta1 = (0.0 + u_le) % nx
    S.susp_fluid_step_noalloc(nx, ny, nz, tau, delta1, u_le, b.data_ptr(), c.data_ptr(),
                              visc.data_ptr(), stream)
    torch.cuda.synchronize()
    s2 = visc.cpu().numpy().reshape(3, 3)
    f1 = b.cpu().numpy().astype(np.float64).reshape(19, nz, ny, nx)
    f2 = c.cpu().numpy().astype(np.float64).reshape(19, nz, ny, nx)

    for got, ref in ((f1, f1_ref), (f2, f2_ref)):
        assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
    for got, ref in ((s1, s1_ref), (s2, s2_ref)):
        assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()


def test_noalloc_rejects_oversized_box():
    from paper_1904_02929_gb300 import susp as S
    with pytest.raises(S.SuspError) as e:
        S.susp_fluid_step_noalloc(512, 8, 256, 1.0, 0.0, 0.0, 16, 16, 16, 0)
    assert e.value.status == S.SUSP_EINVAL


def test_noalloc_rejects_overlapping_buffers():
    """The step reads f_in while writing f_out, so an in-place or partly
    overlapping call is refused before anything is launched."""
    from paper_1904_02929_gb300 import susp as S
    nx, ny, nz = 8, 8, 8
    nbytes = 19 * nx * ny * nz * 4
    base = 1 << 20
    for f_out in (base, base + nbytes - 4, base - nbytes + 4):
        with pytest.raises(S.SuspError) as e:
            S.susp_fluid_step_noalloc(nx, ny, nz, 1.0, 0.0, 0.0, base, f_out, 16, 0)
        assert e.value.status == S.SUSP_EINVAL
