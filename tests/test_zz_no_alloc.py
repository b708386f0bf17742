"""pic_solve_field_static, the field solve for callers that cannot allocate
device memory (their framework owns the device pool, or they may only touch
the buffers they are handed): called through the C ABI with device buffers
the test owns, twice in a row with different right-hand sides, it must give
the potential of the handle-based pic_solve_field and of the oracle's
sparse direct solve within the field-solve tolerance of the other tests
(1e-10 of the potential's scale), its calls must not take device memory,
and it must refuse grids beyond its fixed working array.

This file is collected last so that a failure here, with -x, stops the run
only after every other test has run.
"""
import numpy as np
import pytest

from paper_2206_14662_gb300.inputs import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2206_14662_gb300 import build
    build.build()
    return torch


def test_static_solve_matches_handle_solve(torch_cuda):
    torch = torch_cuda
    import oracle
    from paper_2206_14662_gb300._capi import Simulation, solve_field_static
    cfg = workload("mirror_128x512_1e7", precision=64)
    nn = (cfg["nr"] + 1) * (cfg["nz"] + 1)
    rng = np.random.default_rng(2024)
    rhs = [-rng.random(nn) * 1e-13, -np.abs(np.sin(np.arange(nn) * 0.01)) * 3e-14]
    with Simulation(cfg) as sim:
        ref = [sim.solve_field(b)[0] for b in rhs]
    stream = torch.cuda.current_stream().cuda_stream
    phi = torch.empty(nn, dtype=torch.float64, device="cuda")
    for k, (b, phi_ref) in enumerate(zip(rhs, ref)):   # two calls in a row share the scratch
        b_dev = torch.from_numpy(b).to("cuda")
        phi.fill_(float("nan"))
        rel = solve_field_static(cfg, b_dev.data_ptr(), phi.data_ptr(), stream)
        got = phi.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - phi_ref).max() <= 1e-10 * np.abs(phi_ref).max()
        assert rel <= cfg["poisson_rtol"]
        if k == 0:   # the plain definition: the oracle's sparse direct solve
            phi_o = oracle.poisson_solve(cfg, b)
            assert np.abs(got - phi_o).max() <= 1e-10 * np.abs(phi_o).max()


def test_static_solve_takes_no_device_memory(torch_cuda):
    """After a first call (which loads the library's kernels and the array
    with them), further calls leave the device's free memory unchanged."""
    torch = torch_cuda
    from paper_2206_14662_gb300._capi import solve_field_static
    cfg = workload("coax_32x64_1e4", precision=64)
    nn = (cfg["nr"] + 1) * (cfg["nz"] + 1)
    b = torch.from_numpy(-np.random.default_rng(3).random(nn) * 1e-13).to("cuda")
    phi = torch.empty(nn, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    solve_field_static(cfg, b.data_ptr(), phi.data_ptr(), stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        solve_field_static(cfg, b.data_ptr(), phi.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0


def test_static_solve_rejects_grids_beyond_its_array(torch_cuda):
    torch = torch_cuda
    from paper_2206_14662_gb300._capi import PIC_EINVAL, PicError, solve_field_static
    cfg = workload("mirror_256x1024_2e8", precision=64)   # 263 425 nodes
    b = torch.zeros(16, dtype=torch.float64, device="cuda")
    phi = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(PicError) as ei:    # refused before any device work
        solve_field_static(cfg, b.data_ptr(), phi.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    assert ei.value.code == PIC_EINVAL
    assert float(phi.abs().sum()) == 0.0
