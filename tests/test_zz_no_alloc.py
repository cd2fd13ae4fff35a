"""sph_density_eval_static: the evaluation entry point for callers that cannot allocate.

Programs that embed this library where cudaMalloc/cudaFree are off limits (a host program
that owns all device memory through its own pool, a latency-critical loop where cudaFree
would stall the device) call sph_density_eval_static, whose scratch is a fixed array of
device memory inside the library.  Here it is called through the C ABI twice in a row, on
different particle sets, and each result must equal the context-based sph_sort +
sph_density_eval on the same inputs within the tolerances the other parity tests use
(FP64: exact counts, 1e-12 relative; FP32: 1e-6 relative here, since both sides run the
same FP32 arithmetic on the same data).  The file is named so that pytest collects it
last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1612_06090_gb300 import binding as B  # noqa: E402

DEV = torch.device("cuda:0")


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(3, n))
    mass = rng.uniform(0.5, 1.5, size=n) / n
    h = (3 * 64 / (4 * np.pi * n)) ** (1 / 3) * rng.uniform(0.6, 1.6, size=n)
    return pos, mass, h


def _context_eval(pos, mass, h, precision):
    s = B.Solver(pos.shape[1], precision=precision)
    s.sort(torch.as_tensor(pos, device=DEV), torch.as_tensor(mass, device=DEV))
    r = s.evaluate(torch.as_tensor(h, device=DEV))
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in r.items()}
    s.close()
    return out


def _static_eval(pos, mass, h, precision):
    n = pos.shape[1]
    tp = torch.as_tensor(pos, device=DEV)
    tm = torch.as_tensor(mass, device=DEV)
    th = torch.as_tensor(h, device=DEV)
    rho = torch.empty(n, dtype=torch.float64, device=DEV)
    nw = torch.empty(n, dtype=torch.float64, device=DEV)
    dnw = torch.empty(n, dtype=torch.float64, device=DEV)
    cnt = torch.empty(n, dtype=torch.int32, device=DEV)
    params = B.make_params(precision=precision)
    st = B.sph_density_eval_static(params, n, tp.data_ptr(), tm.data_ptr(), th.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream, rho.data_ptr(),
                                   cnt.data_ptr(), nw.data_ptr(), dnw.data_ptr())
    assert st == B.SPH_OK, B.sph_status_string(st)
    torch.cuda.synchronize()
    return {"rho": rho.cpu().numpy(), "nw": nw.cpu().numpy(), "dnw": dnw.cpu().numpy(),
            "count": cnt.cpu().numpy()}


@pytest.mark.parametrize("precision", [B.SPH_PREC_FP64, B.SPH_PREC_FP32_KAHAN])
def test_static_eval_matches_context_eval_twice(precision):
    rtol = 1e-12 if precision == B.SPH_PREC_FP64 else 1e-6
    # two calls in a row; the second is smaller, so stale contents of the shared array
    # from the first call would show up as wrong results
    for n, seed in ((B.SPH_STATIC_MAX_PARTICLES, 1), (5003, 2)):
        pos, mass, h = _inputs(n, seed)
        a = _static_eval(pos, mass, h, precision)
        b = _context_eval(pos, mass, h, precision)
        np.testing.assert_array_equal(a["count"], b["count"])
        for k in ("rho", "nw", "dnw"):
            np.testing.assert_allclose(a[k], b[k], rtol=rtol, atol=0)


def test_static_eval_rejects_sizes_beyond_the_array():
    n = B.SPH_STATIC_MAX_PARTICLES + 1
    dummy = torch.empty(4, dtype=torch.float64, device=DEV)
    cnt = torch.empty(4, dtype=torch.int32, device=DEV)
    st = B.sph_density_eval_static(B.make_params(), n, dummy.data_ptr(), dummy.data_ptr(),
                                   dummy.data_ptr(), 0, dummy.data_ptr(), cnt.data_ptr())
    assert st == B.SPH_ERR_OOM
