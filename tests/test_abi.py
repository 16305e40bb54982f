"""Host-side checks of the C ABI: the library loads and exports every entry point
declared in include/*.h.  No device work."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names.update(re.findall(r"^RBF_API\s+[\w\s\*]*?\b(rbf_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import paper_1606_07652_gb300 as rbf
    from paper_1606_07652_gb300 import build as b
    b.build()
    return rbf.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("rbf_tree_build", "rbf_fmm_matvec", "rbf_interp_solve", "rbf_tree_free"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    lib.rbf_strerror.restype = ctypes.c_char_p
    assert lib.rbf_strerror(0) == b"success"
    assert lib.rbf_strerror(-1) == b"invalid argument"
    assert lib.rbf_strerror(-4) == b"iterative solve did not converge"


def test_argument_errors_need_no_device(lib):
    """Null pointers are rejected before any CUDA call."""
    out = ctypes.c_void_p()
    assert lib.rbf_tree_build(None, 10, 2, None, 1.0, 2, None, ctypes.byref(out)) == -1
    assert lib.rbf_fmm_matvec(None, 0, 1.0, None, 0, None, 0, None, 0, 1, None) == -1
    assert lib.rbf_tree_get_info(None, None) == -1
    rate = ctypes.c_double(0.0)
    assert lib.rbf_peak_probe(0, ctypes.c_double(0.1), None, None) == -1       # no output
    assert lib.rbf_peak_probe(0, ctypes.c_double(0.0), ctypes.byref(rate), None) == -1
    assert lib.rbf_peak_probe(9, ctypes.c_double(0.1), ctypes.byref(rate), None) == -1  # kind


def test_batch_and_tuning_argument_errors_need_no_device(lib):
    """The batch, cost-model and tuning entry points reject null pointers and
    out-of-range options with RBF_EINVAL before any CUDA call."""
    from paper_1606_07652_gb300 import _lib as L
    P = ctypes.byref
    model = L.CostModel(5e-13, 1e-12, 1e-12, 1e-12, 1e-5)
    params, depth = L.FmmParams(), ctypes.c_int(0)
    err, pred = ctypes.c_double(0.0), ctypes.c_double(0.0)
    # rbf_autotune_cost: no model, then bad eps / tol / N / d / nrhs
    assert lib.rbf_autotune_cost(0, 2.0, 3, 1000, 1, 1.0, 1e-6, None, P(params), P(depth),
                                 P(err), P(pred)) == -1
    for eps, tol, n, d, nrhs in ((0.0, 1e-6, 1000, 3, 1), (2.0, 0.0, 1000, 3, 1),
                                 (2.0, 1e-6, 0, 3, 1), (2.0, 1e-6, 1000, 0, 1),
                                 (2.0, 1e-6, 1000, L.MAX_DIM + 1, 1), (2.0, 1e-6, 1000, 3, 0)):
        assert lib.rbf_autotune_cost(0, eps, d, n, nrhs, 1.0, tol, P(model), P(params), P(depth),
                                     P(err), P(pred)) == -1
    assert lib.rbf_autotune(0, 2.0, 3, 1000, 1.0, 1e-6, None, P(depth), None) == -1
    assert lib.rbf_autotune(0, -1.0, 3, 1000, 1.0, 1e-6, P(params), P(depth), None) == -1
    assert lib.rbf_kernel_error(0, 2.0, 3, None, 1.0, 3, P(err)) == -1
    assert lib.rbf_kernel_error(0, 2.0, 3, P(params), 1.0, 0, P(err)) == -1   # depth 0
    assert lib.rbf_cost_calibrate(None, None) == -1
    # rbf_batch_create_opts: no problems, no output, bad tolerance, unknown choice
    out = ctypes.c_void_p()
    prob = ctypes.create_string_buffer(64)
    opts = L.BatchOpts(1e-6, L.BATCH_AUTO, None)
    assert lib.rbf_batch_create_opts(None, 1, P(opts), None, P(out)) == -1
    assert lib.rbf_batch_create_opts(prob, 0, P(opts), None, P(out)) == -1
    assert lib.rbf_batch_create_opts(prob, 1, None, None, P(out)) == -1
    assert lib.rbf_batch_create_opts(prob, 1, P(L.BatchOpts(0.0, L.BATCH_AUTO, None)), None,
                                     P(out)) == -1
    assert lib.rbf_batch_create_opts(prob, 1, P(L.BatchOpts(1e-6, 7, None)), None, P(out)) == -1
    # operations on a missing batch or tree
    stats, a, b = L.BatchStats(), ctypes.c_double(0.0), ctypes.c_double(0.0)
    shape, total = ctypes.c_int(-1), ctypes.c_int64(0)
    it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
    assert lib.rbf_batch_get_stats(None, P(stats)) == -1
    assert lib.rbf_batch_time_parts(None, 1, 1, P(a), P(b), None) == -1
    assert lib.rbf_batch_layout(None, None, None, None, P(total)) == -1
    assert lib.rbf_batch_matvec(None, 1, None, None, None) == -1
    assert lib.rbf_batch_solve(None, None, None, 30, 100, 1e-8, 1, P(rr), P(it), None, None) == -1
    assert lib.rbf_p2m_launch_shape(None, P(shape)) == -1


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/rbf.h compiles as strict ISO C99 (-pedantic -Werror), and a C
    program taking the address of every declared entry point links against
    librbf.so: the boundary needs no C++ and no torch."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    from paper_1606_07652_gb300 import _lib
    names = _declared()
    src = tmp_path / "abi.c"
    src.write_text('#include "rbf.h"\n#include <stdio.h>\n\nint main(void)\n{\n'
                   "    typedef void (*any_fn)(void);\n    any_fn fns[] = {\n"
                   + ",\n".join(f"        (any_fn){n}" for n in names)
                   + "\n    };\n    printf(\"%d\\n\", (int)(sizeof(fns) / sizeof(fns[0])));\n"
                   "    return 0;\n}\n")
    obj, exe = tmp_path / "abi.o", tmp_path / "abi"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I" + os.path.join(ROOT, "include"), "-c", str(src), "-o", str(obj)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    libdir = os.path.dirname(_lib.library_path())
    r = subprocess.run([gcc, str(obj), "-L" + libdir, "-lrbf",
                        "-Wl,--unresolved-symbols=ignore-in-shared-libs", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
