"""The allocation-free mass/flux entry point (lbm_flux_noalloc) against the
library's regular one (lbm_flux) and against the oracle's flux of the same
stored values.

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


def _stored(f, w, precision, scale):
    """The state in the library's storage form (f - w; FP16: times the
    power-of-two scale, rounded) and its exact FP64 decoding."""
    d = f - w[:, None]
    if precision == "f16s":
        host = (d.astype(np.float32) * np.float32(scale)).astype(np.float16)
        dec = host.astype(np.float64) / scale
    else:
        host = d.astype(np.float64 if precision == "f64" else np.float32)
        dec = host.astype(np.float64)
    return host, w[:, None] + dec


# one block (45,880 nodes); several blocks with a partial last one
# (63 x 65 x 71 = 290,745 nodes: 71 chunks of 4096, the last 4,089)
@pytest.mark.parametrize("dims", [(40, 37, 31), (63, 65, 71)])
@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("layout", ["soa", "aos"])
def test_noalloc_matches_lbm_flux_and_oracle_twice(precision, layout, dims):
    import torch

    from paper_1111_0922_gb300 import build, lbm

    build.build()
    lbm.load()
    torch.cuda.set_device(0)
    per = (1, 1, 1)
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
    host, decoded = _stored(f, w, precision, scale)
    # the oracle's sums of the very values the device holds (FP64 in
    # another order: 1e-12)
    ora = oracle.flux(decoded, (gx, 0.0, 0.0))
    npad = n + 64
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
        out.fill_(np.nan)
        lbm.lbm_flux_noalloc(dev, lbm.PRECISIONS[precision], lbm.LBM_SOA if layout == "soa" else lbm.LBM_AOS,
                             n, npad, scale, gx, out, stream)
        got = out.cpu().numpy()
        for ref in (want, ora):
            assert abs(got[0] - ref[0]) <= tol * abs(ref[0])
            assert abs(got[1] - ref[1]) <= tol * abs(ref[1])
    lat.close()


def test_noalloc_chunk_above_minimum():
    """Past 4096 x 16384 nodes the chunk grows with n (here 4352 nodes, the
    last block partial): FP32 SoA state made on the device, checked against
    FP64 sums by plain PyTorch."""
    import torch

    from paper_1111_0922_gb300 import lbm

    lbm.load()
    torch.cuda.set_device(0)
    n = 4096 * 16384 + 123457
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    d = (torch.rand((19, n), generator=g, device="cuda", dtype=torch.float32) - 0.5) * 2e-3
    gx = 3e-6
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        lbm.lbm_flux_noalloc(d, lbm.LBM_F32, lbm.LBM_SOA, n, n, 1.0, gx, out,
                             torch.cuda.current_stream().cuda_stream)
        got = out.cpu().numpy()
        _, w = oracle.lattice()
        cx = torch.tensor([oracle.lattice()[0][i][0] for i in range(19)], dtype=torch.float64, device="cuda")
        fd = d.double() + torch.tensor(w, device="cuda")[:, None]
        rho = fd.sum(0)
        m = float(rho.sum())
        j = float((cx[:, None] * fd).sum(0).add(0.5 * gx * rho).sum())
        assert abs(got[0] - m) <= 1e-12 * abs(m) and abs(got[1] - j) <= 1e-12 * abs(j)
    del d


def test_noalloc_rejects_oversize():
    import torch

    from paper_1111_0922_gb300 import lbm

    lbm.load()
    dev = torch.zeros(19 * 8, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_flux_noalloc(dev, lbm.LBM_F32, lbm.LBM_AOS, 16384 * 65536 + 1, 0, 1.0, 0.0, out)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
