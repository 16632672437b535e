"""The allocation-free mass/flux entry point (lbm_flux_noalloc) against the
library's regular one (lbm_flux) on the same state.

lbm_flux_noalloc exists for callers that cannot allocate device memory (their
device memory already belongs to a pool, or they cannot afford the device-wide
synchronisation of cudaMalloc/cudaFree); it keeps its scratch in a fixed array
inside the library.  This file is collected last so that a run stopping at the
first failure has run every other test first; it also passes alone."""
import numpy as np
import pytest

import oracle
from paper_1111_0922_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("layout", ["soa", "aos"])
def test_noalloc_matches_lbm_flux_twice(precision, layout):
    import torch

    from paper_1111_0922_gb300 import build, lbm

    build.build()
    lbm.load()
    torch.cuda.set_device(0)
    dims, per = (40, 37, 31), (1, 1, 1)
    n = int(np.prod(dims))
    gx = 1e-5
    rho = inputs.density_noise(dims, seed=9)
    _, w = oracle.lattice()
    f = w[:, None] * rho[None, :]
    f[1] += 2e-4  # a net x momentum
    lat = lbm.Lattice(dims, per, variant="aa", precision=precision, layout=layout,
                      force=(gx, 0.0, 0.0), f16_scale=2.0 ** 14)
    lat.set_geometry(None)
    lat.set_pdfs(f)
    want = lat.flux()
    scale = lat.info.f16_scale
    # the same state as the caller's own device array in storage form
    d = f - w[:, None]
    npad = n + 64
    if precision == "f16s":
        # the library's encoding: f - w in FP32, times the power-of-two scale, to FP16
        host = (d.astype(np.float32) * np.float32(scale)).astype(np.float16)
    else:
        host = d.astype(np.float64 if precision == "f64" else np.float32)
    if layout == "soa":
        arr = np.zeros((19, npad), host.dtype)
        arr[:, :n] = host
    else:
        arr = np.ascontiguousarray(host.T)
    dev = torch.from_numpy(arr).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    tol = 1e-12  # same decoded values, FP64 sums in another order
    for _ in range(2):  # two calls in a row share the scratch
        out.zero_()
        lbm.lbm_flux_noalloc(dev, lbm.PRECISIONS[precision], lbm.LBM_SOA if layout == "soa" else lbm.LBM_AOS,
                             n, npad, scale, gx, out, stream)
        got = out.cpu().numpy()
        assert abs(got[0] - want[0]) <= tol * abs(want[0])
        assert abs(got[1] - want[1]) <= tol * abs(want[1])
    lat.close()


def test_noalloc_rejects_oversize():
    import torch

    from paper_1111_0922_gb300 import lbm

    lbm.load()
    dev = torch.zeros(19 * 8, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_flux_noalloc(dev, lbm.LBM_F32, lbm.LBM_AOS, 16384 * 65536 + 1, 0, 1.0, 0.0, out)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
