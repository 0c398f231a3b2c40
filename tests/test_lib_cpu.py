"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, and exports every entry point that include/grest.h declares;
the ctypes structures match the header's layout."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_19439_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def header_functions():
    src = open(os.path.join(ROOT, "include", "grest.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grest_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    """The ctypes binding declares exactly the header's entry points."""
    from paper_2603_19439_gb300 import grest
    assert sorted(grest.EXPORTS) == header_functions()


def test_status_strings_and_defaults(lib):
    from paper_2603_19439_gb300 import grest
    L = grest.load_library()
    assert L.grest_status_str(0) == b"ok"
    assert L.grest_status_str(2) == b"invalid update batch"
    cfg = grest.default_config(16)
    assert (cfg.k, cfg.L, cfg.P, cfg.op, cfg.subspace) == (16, 100, 100, grest.OP_ADJ, grest.SUB_AUTO)
    assert cfg.drop_tol == 1e-7


def test_struct_sizes_match_header():
    from paper_2603_19439_gb300 import grest
    # int32 x 9, pad, uint64, double, int64 x 3
    assert ctypes.sizeof(grest.Config) == 40 + 8 + 8 + 24
    assert ctypes.sizeof(grest.Update) == 8 * 10 + 8
    # ..., prof_* per class (5), kernel_launches, prof_bytes, prof_kind_* (10 kinds x 4)
    assert ctypes.sizeof(grest.Stats) == 24 + 24 + 48 + 32 + 3 * 40 + 8 + 40 + 4 * 80


def test_struct_sizes_match_a_c_compiler(tmp_path):
    """The ctypes layouts against sizeof() from a C compiler reading the header."""
    import shutil
    import subprocess
    from paper_2603_19439_gb300 import grest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "grest.h"\n'
                   'int main(void) { printf("%zu %zu %zu\\n", sizeof(grest_config), sizeof(grest_update), '
                   'sizeof(grest_stats)); return 0; }\n')
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert [int(x) for x in out] == [ctypes.sizeof(grest.Config), ctypes.sizeof(grest.Update),
                                     ctypes.sizeof(grest.Stats)]


def test_init_rejects_bad_arguments_without_gpu(lib):
    """Argument checks happen on the host before any device call."""
    import numpy as np
    from paper_2603_19439_gb300 import grest
    L = grest.load_library()
    cfg = grest.default_config(0)
    h = ctypes.c_void_p()
    rp = np.array([0, 0], np.int64)
    assert L.grest_init(ctypes.byref(cfg), 1, rp.ctypes.data, None, None, None, None, None, ctypes.byref(h)) == 1
    cfg = grest.default_config(2, L=200, P=100)
    assert L.grest_init(ctypes.byref(cfg), 1, rp.ctypes.data, None, None, None, None, None, ctypes.byref(h)) == 1


def test_init_rejects_unsupported_modes_without_gpu(lib):
    """The explicit Delta of DELTA / LOWRANK exists for ADJ and LAP; LOWRANK has
    no mixed-precision refinement.  These are refused before any device call."""
    import numpy as np
    from paper_2603_19439_gb300 import grest
    L = grest.load_library()
    h = ctypes.c_void_p()
    rp = np.array([0, 0, 0], np.int64)
    u0 = np.eye(2)
    t0 = np.ones(2)
    for kw in (dict(op=grest.OP_NLAP, projection=grest.PROJ_LOWRANK), dict(op=grest.OP_NLAP, w_block=grest.WB_DELTA),
               dict(precision=grest.MIXED, projection=grest.PROJ_LOWRANK)):
        cfg = grest.default_config(1, **kw)
        st = L.grest_init(ctypes.byref(cfg), 2, rp.ctypes.data, None, None, u0.ctypes.data, t0.ctypes.data, None,
                          ctypes.byref(h))
        assert st == 8, (kw, st)
    cfg = grest.default_config(1, projection=7)
    assert L.grest_init(ctypes.byref(cfg), 2, rp.ctypes.data, None, None, u0.ctypes.data, t0.ctypes.data, None,
                        ctypes.byref(h)) == 1


def test_batch_create_checks_arguments_without_gpu(lib):
    """grest_batch_create only records the context handles: argument checks
    (empty, NULL entry, the same context twice) run on the host.  Status 1 is
    GREST_ERR_INVALID_ARG."""
    from paper_2603_19439_gb300 import grest
    L = grest.load_library()
    vp = ctypes.c_void_p
    h = vp()
    fake = (vp * 3)(0x1000, 0x2000, 0x1000)
    assert L.grest_batch_create(0, fake, 1, ctypes.byref(h)) == 1
    assert L.grest_batch_create(3, fake, 2, ctypes.byref(h)) == 1  # duplicate
    nul = (vp * 2)(0x1000, None)
    assert L.grest_batch_create(2, nul, 2, ctypes.byref(h)) == 1
    assert L.grest_batch_create(2, fake, 0, ctypes.byref(h)) == 1
    assert L.grest_batch_create(2, fake, 4, ctypes.byref(h)) == 0 and h.value
    assert L.grest_batch_apply_updates(None, None, None, None) == 1
    L.grest_batch_destroy(h)


def test_checkpoint_calls_check_arguments_without_gpu(lib):
    """A byte array that is not a checkpoint (wrong tag, too short) is
    rejected on the host before any device work, by grest_restore and by the
    host reader grest_checkpoint_embedding; NULL handles are rejected too.
    Status 1 is GREST_ERR_INVALID_ARG."""
    from paper_2603_19439_gb300 import grest
    L = grest.load_library()
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    junk = (ctypes.c_uint8 * 4096)(*([7] * 4096))
    h, n, k, nb = vp(), i64(), i32(), i64()
    assert L.grest_restore(junk, 4096, None, ctypes.byref(h)) == 1 and not h.value
    assert L.grest_restore(junk, 3, None, ctypes.byref(h)) == 1
    assert L.grest_restore(None, 0, None, ctypes.byref(h)) == 1
    assert L.grest_checkpoint_embedding(junk, 4096, None, None, None, ctypes.byref(n), ctypes.byref(k)) == 1
    assert L.grest_checkpoint_embedding(junk, 4096, None, None, None, None, None) == 1
    assert L.grest_checkpoint(None, None, ctypes.byref(nb)) == 1
    assert L.grest_server_set_eviction(None, 1) == 1
    assert L.grest_server_counters(None, None, None, None) == 1
    with pytest.raises(grest.GrestError):
        grest.checkpoint_embedding(bytes(junk))


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/grest.h compiles as C99 with warnings as errors, and a C
    program links against libgrest.so and calls the host-only entry points
    (defaults, status strings, argument checks) without a GPU."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "grest.h"
int main(void) {
  grest_config cfg;
  if (grest_config_default(&cfg, 16) != GREST_OK) return 1;
  if (cfg.k != 16 || cfg.L != 100 || cfg.P != 100 || cfg.precision != GREST_FP64) return 2;
  if (strcmp(grest_status_str(GREST_OK), "ok") != 0) return 3;
  grest_ctx *ctx = NULL;
  if (grest_init(NULL, 0, NULL, NULL, NULL, NULL, NULL, NULL, &ctx) != GREST_ERR_INVALID_ARG || ctx) return 4;
  if (grest_restore(NULL, 0, NULL, &ctx) != GREST_ERR_INVALID_ARG) return 5;
  printf("abi ok\n");
  return 0;
}
''')
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib._name)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", libdir, "-lgrest", f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "abi ok", (r.returncode, r.stdout, r.stderr)


def test_null_handles_rejected_without_gpu(lib):
    """Every entry point that takes a context, batch or server handle returns
    GREST_ERR_INVALID_ARG (1) for NULL before any device work, and the
    destroy calls accept NULL."""
    from paper_2603_19439_gb300 import grest
    L = grest.load_library()
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    n, m, t, d = i64(), i32(), i64(), i32()
    st = grest.Stats()
    u = grest.Update()
    assert L.grest_apply_update(None, ctypes.byref(u), None) == 1
    assert L.grest_sync(None) == 1
    assert L.grest_get_embedding(None, None, None, None, ctypes.byref(n), 0) == 1
    assert L.grest_set_embedding(None, None, None, 0) == 1
    assert L.grest_get_ritz_values(None, None, ctypes.byref(m)) == 1
    assert L.grest_get_stats(None, ctypes.byref(st)) == 1
    assert L.grest_centrality(None, 0, None, None, None, 0) == 1
    assert L.grest_apply_operator(None, None, 1, None, 1, 1) == 1
    assert L.grest_gram(None, None, 1, 1, None, 1, 1, 1, None, 1) == 1
    assert L.grest_gram_f32(None, None, 1, 1, None, 1, 1, 1, None, 1) == 1
    assert L.grest_gemm_f32(None, 1, 1, 1, 1.0, None, 1, None, 1, 0.0, None, 1, None, 1) == 1
    assert L.grest_gram_noalloc(None, 1, 1, None, 1, 1, 1, None, 1, None) == 1
    assert L.grest_get_device_bytes(None, ctypes.byref(n)) == 1
    assert L.grest_batch_apply_updates(None, None, None, None) == 1
    assert L.grest_server_create(0, 0, ctypes.byref(ctypes.c_void_p())) == 1
    assert L.grest_server_add_graph(None, None, 1, None, None, None, None, None, ctypes.byref(d)) == 1
    assert L.grest_server_submit(None, 0, ctypes.byref(u), ctypes.byref(t)) == 1
    assert L.grest_server_wait(None, 0, None, None, None, None) == 1
    assert L.grest_server_poll(None, 0, ctypes.byref(d)) == 1
    assert L.grest_server_remove_graph(None, 0) == 1
    assert L.grest_server_get_embedding(None, 0, None, None, None, ctypes.byref(n)) == 1
    assert L.grest_server_resident(None, None, None) == 1
    L.grest_destroy(None)
    L.grest_batch_destroy(None)
    L.grest_server_destroy(None)


def test_gram_bindings_reject_bad_tensors_before_the_library():
    """grest_gram / grest_gram_f32 / grest_gram_noalloc take raw pointers, so
    the binding checks shapes, dtypes, strides and the device before the
    call: a short Y or a small C would otherwise be read or written out of
    bounds on the GPU."""
    torch = pytest.importorskip("torch")
    from paper_2603_19439_gb300 import grest
    f64 = torch.float64
    X, Y, C = torch.zeros((50, 4), dtype=f64), torch.zeros((50, 3), dtype=f64), torch.zeros((4, 3), dtype=f64)
    grest.check_gram_args(X, Y, C, "float64", "t", require_cuda=False)  # well formed
    bad = [
        (X, torch.zeros((49, 3), dtype=f64), C),            # Y shorter than X
        (X, Y, torch.zeros((3, 3), dtype=f64)),             # C has fewer rows than X has columns
        (X, Y, torch.zeros((4, 2), dtype=f64)),             # C has fewer columns than Y
        (X.float(), Y, C),                                  # dtype
        (X, Y, C.float()),                                  # output dtype
        (X.t(), torch.zeros((4, 3), dtype=f64), C),         # inner stride != 1
        (X[:, None, :], Y, C),                              # not 2-D
        (torch.zeros((0, 4), dtype=f64), torch.zeros((0, 3), dtype=f64), C),  # no rows
    ]
    for args in bad:
        with pytest.raises(grest.GrestError) as e:
            grest.check_gram_args(*args, "float64", "t", require_cuda=False)
        assert e.value.code == 1
    # host tensors are rejected by the public wrappers (a CUDA device is required)
    with pytest.raises(grest.GrestError) as e:
        grest.gram_noalloc(X, Y, C)
    assert e.value.code == 1
    with pytest.raises(grest.GrestError) as e:
        grest.check_gram_args(X.float(), Y.float(), C, "float32", "grest_gram_f32")
    assert e.value.code == 1


def test_group_create_rejects_bad_arguments_without_gpu(lib):
    """grest_group_create checks its arguments on the host before any device
    call: no graphs, null arrays, a capacity factor below 1, a buffer that is
    not a checkpoint."""
    import numpy as np
    from paper_2603_19439_gb300 import grest
    L = grest.load_library()
    h = ctypes.c_void_p()
    junk = np.zeros(256, np.uint8)
    ptrs = (ctypes.c_void_p * 1)(junk.ctypes.data)
    sizes = (ctypes.c_int64 * 1)(junk.size)
    assert L.grest_group_create(0, ptrs, sizes, 1.25, ctypes.byref(h)) == 1
    assert L.grest_group_create(1, None, sizes, 1.25, ctypes.byref(h)) == 1
    assert L.grest_group_create(1, ptrs, sizes, 0.5, ctypes.byref(h)) == 1
    assert L.grest_group_create(1, ptrs, sizes, 1.25, ctypes.byref(h)) == 1  # not a checkpoint
    assert h.value is None
    assert L.grest_group_apply_updates(None, None, None, None) == 1
    assert L.grest_group_info(None, None, None, None, None, None, None) == 1
    L.grest_group_destroy(None)


def test_embedding_async_checks_buffers_before_any_device_call():
    """Tracker.embedding_async rejects a U buffer with too few rows or the
    wrong width, and a short theta buffer, on the host, before the library
    is called (a short buffer would be written past its end by the device)."""
    import numpy as np
    from paper_2603_19439_gb300 import grest

    class NoLib:
        def __getattr__(self, name):
            raise AssertionError("the library must not be called")

    tr = grest.Tracker.__new__(grest.Tracker)
    tr.lib, tr.h, tr.k, tr.n = NoLib(), None, 4, 100
    with pytest.raises(ValueError):
        tr.embedding_async(np.zeros((99, 4)), np.zeros(4))
    with pytest.raises(ValueError):
        tr.embedding_async(np.zeros((100, 3)), np.zeros(4))
    with pytest.raises(ValueError):
        tr.embedding_async(np.zeros((100, 4)), np.zeros(3))
