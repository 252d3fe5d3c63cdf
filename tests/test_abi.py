"""CPU checks of the C ABI boundary: the library builds, loads, exports every
function include/cwt.h declares, and validates arguments on the host before
touching a device.  No transform is computed here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cwt():
    import paper_2302_03909_gb300 as pkg
    pkg.load_library()
    return pkg


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cwt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cwt_[a-z_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for required in ["cwt_plan_create", "cwt_exec", "cwt_wavelet_power", "cwt_plan_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(cwt):
    lib = cwt.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(cwt.ABI_FUNCTIONS) == declared_functions()


def test_status_strings(cwt):
    assert cwt.cwt_status_string(0) == "ok"
    assert "argument" in cwt.cwt_status_string(1)
    assert cwt.cwt_status_string(99) == "unknown status"


def test_paper_grid_matches_sec_3_1(cwt):
    # w~ = w~_min 2^{i + j/N_subs}, w~_min = c_w pi / N, N_levs = Nint(log2 N)
    N, n_subs = 1000, 3
    g = cwt.cwt_scales_paper_grid(N, "gdw", 6.0, n_subs)
    n_levs = round(math.log2(N))
    assert len(g) == n_levs * n_subs
    cw = 2 / math.sqrt(5)
    assert g[0] == pytest.approx(cw * math.pi / N, rel=1e-15)
    assert np.allclose(g[1:] / g[:-1], 2 ** (1 / n_subs), rtol=1e-13)
    gm = cwt.cwt_scales_paper_grid(N, "morlet", 6.0, n_subs)
    assert gm[0] == pytest.approx(2 / (6 + math.sqrt(38)) * math.pi / N, rel=1e-15)


@pytest.mark.parametrize("kwargs,status", [
    (dict(N=1, scales=[2.0]), 1),
    (dict(N=64, scales=[]), 1),
    (dict(N=64, scales=[2.0, -1.0]), 1),
    (dict(N=64, scales=[2.0, float("nan")]), 1),
    (dict(N=64, scales=[2.0, float("inf")]), 1),
    (dict(N=64, scales=[2.0], dx=0.0), 1),
    (dict(N=64, scales=[2.0], eps_trunc=-1.0), 1),
    (dict(N=64, scales=[2.0], wavelet="morlet", omega0=0.0), 1),
    # periodic, N not 2^k, rows of the Bluestein form (other wavelets, spectrum at the
    # Nyquist frequency): FFT length 2^ceil(log2(2N - 1)) above 2^25
    (dict(N=(1 << 24) + 1, scales=[2.0], boundary="periodic", wavelet="cbsw"), 2),
    (dict(N=(1 << 24) + 1, scales=[0.5], boundary="periodic"), 2),
    (dict(N=64, scales=[2.0], boundary="zero", fft_len=32), 1),   # shorter than N
    (dict(N=64, scales=[2.0], boundary="zero", fft_len=96), 2),   # not 2^k
    (dict(N=64, scales=[2.0], boundary="periodic", fft_len=128), 1),
    (dict(N=1 << 26, scales=[2.0], boundary="zero"), 2),          # M > 2^25
    (dict(N=64, scales=[2.0], min_ctas=-1), 1),
    (dict(N=64, scales=[2.0], wide_batch_bytes=-5), 1),
    (dict(N=64, scales=[2.0], band_depth=3), 1),
    (dict(N=64, scales=[2.0], band_depth=32), 1),
    (dict(N=64, scales=[2.0], wide2_kernel=3), 1),
    (dict(N=64, scales=[2.0], wide2_kernel=-1), 1),
    (dict(N=64, scales=[2.0], scratch="caller", tune=True), 1),     # a tuned plan runs itself
])
def test_plan_argument_checks(cwt, kwargs, status):
    kw = dict(kwargs)
    N, scales = kw.pop("N"), kw.pop("scales")
    with pytest.raises(cwt.CwtError) as e:
        cwt.cwt_plan_create(N, scales, **kw)
    assert e.value.status == status


def test_null_plan_pointers_rejected(cwt):
    lib = cwt.load_library()
    assert lib.cwt_exec(None, None, None, None) == 1
    assert lib.cwt_wavelet_power(None, None, None, None) == 1
    assert lib.cwt_plan_create(None, 64, None, 1, 0, 0) == 1
    assert lib.cwt_plan_destroy(None) == 0
    n = ctypes.c_int32()
    assert lib.cwt_scales_paper_grid(1, 0, 6.0, 2, None, ctypes.byref(n)) == 1


def test_batch_and_options_entry_points_check_their_arguments(cwt):
    """Checked on the host before any CUDA call, so this runs without a GPU."""
    lib = cwt.load_library()
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 1)()
    assert lib.cwt_batch_create(None, arr, arr, arr, None, 1, 1) == 1
    assert lib.cwt_batch_create(ctypes.byref(h), None, arr, arr, None, 1, 1) == 1
    assert lib.cwt_batch_create(ctypes.byref(h), arr, arr, arr, None, 0, 1) == 1          # n < 1
    assert lib.cwt_batch_create(ctypes.byref(h), arr, arr, arr, None, 1, 1) == 1          # NULL plan
    assert h.value is None
    assert lib.cwt_batch_exec(None, None) == 1
    assert lib.cwt_batch_info(None, None, None, None, None) == 1
    assert lib.cwt_batch_destroy(None) == 0
    assert lib.cwt_plan_get_opts(None, None) == 1
    n = ctypes.c_size_t()
    assert lib.cwt_plan_scratch_bytes(None, ctypes.byref(n)) == 1
    o = cwt._Opts()
    lib.cwt_plan_opts_default(ctypes.byref(o))
    o.scratch = 2                                                  # neither cwt_scratch_mode
    sc = (ctypes.c_double * 1)(2.0)
    assert lib.cwt_plan_create_ex(ctypes.byref(h), 64, sc, 1, 0, 0, ctypes.byref(o)) == 1
    assert lib.cwt_exec_scratch(None, None, None, None, None, 0, None) == 1
    with pytest.raises(ValueError):
        cwt.cwt_batch_create([])


def test_plan_options_struct_matches_the_header(cwt):
    """The binding's mirror of cwt_plan_opts has the header's field order and
    the defaults the library fills in."""
    o = cwt._Opts()
    cwt.load_library().cwt_plan_opts_default(ctypes.byref(o))
    assert ctypes.sizeof(o) == 72
    assert (o.omega0, o.dx, o.scale_unit, o.input_dtype, o.fft_len) == (6.0, 1.0, 0, 0, 0)
    assert (o.eps_trunc, o.min_ctas, o.tune, o.wide_batch_bytes) == (1e-10, 0, 0, 0)
    assert (o.precision, o.band_depth, o.wide2_kernel, o.scratch) == (0, 0, 0, 0)
    with open(os.path.join(ROOT, "include", "cwt.h")) as fh:
        text = fh.read()
    body = text[text.index("typedef struct {", text.index("cwt_input_dtype;")):text.index("} cwt_plan_opts;")]
    fields = re.findall(r"^\s+(?:double|int32_t|int64_t)\s+(\w+);", body, flags=re.M)
    assert fields == [name for name, _ in cwt._Opts._fields_]


def test_precision_option_range_checked_on_the_host(cwt):
    """cwt_precision values outside FP32 .. BF16X3 are refused before any CUDA call."""
    lib = cwt.load_library()
    o = cwt._Opts()
    lib.cwt_plan_opts_default(ctypes.byref(o))
    sc = (ctypes.c_double * 1)(4.0)
    h = ctypes.c_void_p()
    for bad in (-1, 5):
        o.precision = bad
        assert lib.cwt_plan_create_ex(ctypes.byref(h), 1024, sc, 1, 0, 0, ctypes.byref(o)) == 1
        assert h.value is None
    assert cwt.PRECISIONS == {"fp32": 0, "fp16": 1, "bf16": 2, "fp16x3": 3, "bf16x3": 4}
