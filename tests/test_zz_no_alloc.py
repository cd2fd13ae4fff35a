"""sph_density_eval_static: the evaluation entry point for callers that cannot allocate.

Programs that embed this library where cudaMalloc/cudaFree are off limits (a host program
that owns all device memory through its own pool, a latency-critical loop where cudaFree
would stall the device) call sph_density_eval_static, whose scratch is a fixed array of
device memory inside the library.  Here it is called through the C ABI:
  - twice in a row, on different particle sets, and each result must equal the
    context-based sph_sort + sph_density_eval on the same inputs within the tolerances the
    other parity tests use (FP64: exact counts, 1e-12 relative; FP32: 1e-6 relative here,
    since both sides run the same FP32 arithmetic on the same data);
  - against the FP64 oracle directly (FP64: exact counts, 1e-12; FP32: 1e-5, counts within
    the pairs the oracle finds within 1e-6 h of the boundary);
  - with a bad position, mass or h, which must come back as SPH_ERR_DEVICE_STATUS before any
    density pass runs, after which a valid call must again match the context path (the
    shared array's state word is cleared by every call).
The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from tests.parity import check_eval

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


def _static_call(pos, mass, h, precision):
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
    torch.cuda.synchronize()
    return st, {"rho": rho.cpu().numpy(), "nw": nw.cpu().numpy(), "dnw": dnw.cpu().numpy(),
                "count": cnt.cpu().numpy()}


def _static_eval(pos, mass, h, precision):
    st, out = _static_call(pos, mass, h, precision)
    assert st == B.SPH_OK, B.sph_status_string(st)
    return out


def _assert_matches_context(a, b, precision):
    rtol = 1e-12 if precision == B.SPH_PREC_FP64 else 1e-6
    np.testing.assert_array_equal(a["count"], b["count"])
    for k in ("rho", "nw", "dnw"):
        np.testing.assert_allclose(a[k], b[k], rtol=rtol, atol=0)


@pytest.mark.parametrize("precision", [B.SPH_PREC_FP64, B.SPH_PREC_FP32_KAHAN])
def test_static_eval_matches_context_eval_twice(precision):
    # two calls in a row; the second is smaller, so stale contents of the shared array
    # from the first call would show up as wrong results
    for n, seed in ((B.SPH_STATIC_MAX_PARTICLES, 1), (5003, 2)):
        pos, mass, h = _inputs(n, seed)
        _assert_matches_context(_static_eval(pos, mass, h, precision),
                                _context_eval(pos, mass, h, precision), precision)


@pytest.mark.parametrize("precision", [B.SPH_PREC_FP64, B.SPH_PREC_FP32_KAHAN])
def test_static_eval_matches_oracle(precision):
    pos, mass, h = _inputs(6000, 3)
    g = _static_eval(pos, mass, h, precision)
    if precision == B.SPH_PREC_FP64:
        check_eval(g, oracle.evaluate(pos, mass, h), rtol=1e-12, count_exact=True)
    else:
        o = oracle.evaluate(pos, mass, h, near_rel=1e-6)
        check_eval(g, o, rtol=1e-5, count_exact=False, near=o["near"], dnw_rtol=1e-4)


def test_static_eval_rejects_bad_input_before_the_pass_and_recovers():
    pos, mass, h = _inputs(3000, 4)
    bad_cases = []
    p = pos.copy()
    p[1, 17] = np.nan
    bad_cases.append((p, mass, h))
    m = mass.copy()
    m[5] = 0.0
    bad_cases.append((pos, m, h))
    for bad_h in (0.5, 0.75, np.nan, -1.0, 0.0):
        hh = h.copy()
        hh[11] = bad_h
        bad_cases.append((pos, mass, hh))
    for prec in (B.SPH_PREC_FP64, B.SPH_PREC_FP32_KAHAN):
        for pp, mm, hh in bad_cases:
            st, _ = _static_call(pp, mm, hh, prec)
            assert st == B.SPH_ERR_DEVICE_STATUS, B.sph_status_string(st)
        # the next valid call starts from a cleared state word
        _assert_matches_context(_static_eval(pos, mass, h, prec), _context_eval(pos, mass, h, prec), prec)


def test_static_eval_rejects_sizes_beyond_the_array():
    n = B.SPH_STATIC_MAX_PARTICLES + 1
    dummy = torch.empty(4, dtype=torch.float64, device=DEV)
    cnt = torch.empty(4, dtype=torch.int32, device=DEV)
    st = B.sph_density_eval_static(B.make_params(), n, dummy.data_ptr(), dummy.data_ptr(),
                                   dummy.data_ptr(), 0, dummy.data_ptr(), cnt.data_ptr())
    assert st == B.SPH_ERR_OOM
