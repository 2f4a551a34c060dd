"""GPU test of lb_step_fp64_static, the step entry point that allocates
nothing (for callers that may not allocate device memory where they step a
lattice; its scratch is a fixed array inside the library).

It is called twice in a row through the C ABI on buffers the test owns and
must reproduce, bit for bit (the tolerance of every binary64 test here), the
states lb_step reaches after one and two steps.  Kept in its own file so it
runs after every other test."""
import numpy as np
import pytest

import lbinputs as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_23647_gb300")


@pytest.mark.parametrize("lattice,shape,stencil,tau,G", [
    ("D2Q9", (61, 47), L.E8_2D, 0.8, -5.0),
    ("D3Q19", (24, 20, 18), L.E8_3D, 1.0, -4.0),
])
def test_static_step_matches_lb_step_on_two_calls(lattice, shape, stencil, tau, G):
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    rho = L.tanh_sphere(nx, ny, nz, min(nx, ny) / 4.0, 1.9, 0.15, 2.0)
    lat = P.Lattice(lattice, shape, rho, stencil.bases, stencil.weights, precision="fp64",
                    tau=tau, G=G)
    f0 = lat.state()
    lat.step(1)
    f1 = lat.state()
    lat.step(1)
    f2 = lat.state()
    lat.close()

    dim = 2 if lattice == "D2Q9" else 3
    vec, w, _ = P.lb_expand_stencil(dim, stencil.bases, stencil.weights)
    params = P.make_params(lattice, shape, "fp64", tau, G)
    dev = torch.device("cuda", 0)
    a = torch.tensor(f0.reshape(f0.shape[0], -1), dtype=torch.float64, device=dev)
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    stream = torch.cuda.current_stream(dev).cuda_stream
    P.lb_step_fp64_static(params, vec, w, a.data_ptr(), b.data_ptr(), stream)
    P.lb_step_fp64_static(params, vec, w, b.data_ptr(), c.data_ptr(), stream)
    torch.cuda.synchronize()
    assert np.array_equal(b.cpu().numpy().reshape(f1.shape), f1)
    assert np.array_equal(c.cpu().numpy().reshape(f2.shape), f2)


def test_static_step_rejects_lattices_beyond_the_scratch():
    params = P.make_params("D2Q9", (2048, 1024), "fp64", 1.0, -5.0)   # 2^21 nodes
    vec, w, _ = P.lb_expand_stencil(2, L.E4_2D.bases, L.E4_2D.weights)
    with pytest.raises(P.LbError) as ei:
        P.lb_step_fp64_static(params, vec, w, 16, 32)
    assert ei.value.status == P.LB_EINVAL
    assert "exceed the fixed scratch" in str(P._lib.lb_last_cuda_error().decode())
