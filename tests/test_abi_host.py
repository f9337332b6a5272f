"""Host-side logic of the C-ABI, on the CPU: buffer layout, packed widths, weight counts and
the argument checks that return before any device work (include/hmpcg.h documents each).

None of these calls touches device memory: the system layout only computes pointers into a
caller-supplied address, and every rejected call returns before its first CUDA call.
"""
import ctypes as C
import math

import pytest

import inputs
import paper_2605_13343_gb300 as h

FAKE_BASE = 1 << 32   # 256-byte aligned address; the layout computes pointers only


@pytest.fixture(autouse=True, scope="module")
def _built():
    import os
    if not os.path.exists(h.LIB_PATH):
        from paper_2605_13343_gb300 import build
        build.build()


def _dims(d):
    return (C.c_int32 * 3)(*(list(d) + [1] * (3 - len(d))))


def _layout(d, base=FAKE_BASE):
    s = h.SystemStruct()
    rc = h.lib().hmpcg_system_layout(len(d), _dims(d), C.c_void_p(base), C.byref(s))
    return rc, s


@pytest.mark.parametrize("d", [(32, 32), (32, 16, 16), (128, 128), (16, 8, 8), (4, 4)])
def test_system_layout_arrays_are_aligned_disjoint_and_inside_the_buffer(d):
    n = math.prod(d)
    nbytes = h.lib().hmpcg_system_bytes(len(d), _dims(d))
    rc, s = _layout(d)
    assert rc == h.OK
    assert s.n == n and s.ndim == len(d)
    assert tuple(s.dims) == tuple(list(d) + [1] * (3 - len(d)))
    arrays = ([(s.diag, 8)] + [(s.wplus[a], 8) for a in range(3)] + [(s.diag32, 4)]
              + [(s.wplus32[a], 4) for a in range(3)] + [(s.rho, 8), (s.perm, 4)])
    spans = sorted((p, p + esz * n) for p, esz in arrays)
    assert spans[0][0] == FAKE_BASE
    for lo, hi in spans:
        assert lo % 256 == 0, "every array starts on a 256-byte boundary"
        assert FAKE_BASE <= lo and hi <= FAKE_BASE + nbytes
    for (_, hi), (lo, _) in zip(spans, spans[1:]):
        assert hi <= lo, "arrays overlap"


@pytest.mark.parametrize("d", [(30, 32), (32, 0), (64,), (8, 8, 8, 8), (0, 0, 0)])
def test_system_layout_rejects_unsupported_grids(d):
    nd = len(d)
    arr = (C.c_int32 * max(3, nd))(*(list(d) + [1] * (max(3, nd) - nd)))
    assert h.lib().hmpcg_system_bytes(nd, arr) == -1
    s = h.SystemStruct()
    assert h.lib().hmpcg_system_layout(nd, arr, C.c_void_p(FAKE_BASE), C.byref(s)) == h.E_INVALID


def test_system_layout_rejects_misaligned_and_null_arguments():
    rc, _ = _layout((32, 32), FAKE_BASE + 16)
    assert rc == h.E_INVALID
    s = h.SystemStruct()
    assert h.lib().hmpcg_system_layout(2, _dims((32, 32)), None, C.byref(s)) == h.E_INVALID
    assert h.lib().hmpcg_system_layout(2, _dims((32, 32)), C.c_void_p(FAKE_BASE), None) == h.E_INVALID
    assert h.lib().hmpcg_system_layout(2, None, C.c_void_p(FAKE_BASE), C.byref(s)) == h.E_INVALID


@pytest.mark.parametrize("cfg", [dict(d=128, n_layers=4, n_heads=4, d_mlp=512, leaf=64, rank=16),
                                 dict(d=64, n_layers=1, n_heads=2, d_mlp=64, leaf=64, rank=16),
                                 dict(d=96, n_layers=2, n_heads=3, d_mlp=256, leaf=64, rank=32)])
def test_weight_count_matches_the_documented_blob_layout(cfg):
    want = sum(math.prod(shape) for _, shape in inputs.network_layout(**cfg))
    c = h.Config(max_n=4096, max_batch=1, max_nrhs=1, leaf=cfg["leaf"], rank=cfg["rank"], d_model=cfg["d"],
                 n_layers=cfg["n_layers"], n_heads=cfg["n_heads"], d_mlp=cfg["d_mlp"])
    assert h.lib().hmpcg_weight_count(C.byref(c)) == want
    assert h.lib().hmpcg_weight_count(None) == -1


@pytest.mark.parametrize("n,leaf,rank", [(1024, 64, 16), (8192, 64, 16), (16384, 64, 32), (4096, 32, 8),
                                         (2 ** 22, 64, 16)])
def test_packed_widths_follow_the_tile_counts(n, leaf, rank):
    k = n // leaf
    levels = int(math.log2(k))
    core = k * leaf * leaf + (k - 1) * rank * rank       # K leaf blocks, K-1 tiles
    assert h.packed_width(n, leaf, rank, h.PRE_LEARNED) == core + 2 * n * rank + n
    assert h.packed_width(n, leaf, rank, h.PRE_SVDH) == core + levels * n * rank
    assert h.packed_width(n, leaf, rank, h.PRE_JACOBI) == -1
    assert h.packed_width(n + 1, leaf, rank, h.PRE_LEARNED) == -1
    assert h.packed_width(n, 0, rank, h.PRE_LEARNED) == -1
    assert h.packed_width(n, leaf, 0, h.PRE_SVDH) == -1


def test_create_rejects_bad_configurations_before_any_device_work():
    out = C.c_void_p(12345)
    for kw in (dict(max_n=1, leaf=64, rank=16), dict(max_n=1024, leaf=0, rank=16),
               dict(max_n=1024, leaf=64, rank=0), dict(max_n=-8, leaf=64, rank=16)):
        c = h.Config(max_batch=1, max_nrhs=1, d_model=128, n_layers=4, n_heads=4, d_mlp=512, **kw)
        assert h.lib().hmpcg_create(C.byref(out), C.byref(c), None, 0, None) == h.E_INVALID
        assert out.value is None, "the handle is cleared on failure"
        out = C.c_void_p(12345)


def test_assemble_and_spmv_argument_checks():
    lib = h.lib()
    rc, s = _layout((32, 16, 16))
    assert rc == h.OK
    rho = C.c_void_p(FAKE_BASE)
    assert lib.hmpcg_assemble(rho, C.byref(s), 7, h.FACE_INV_RHO, None) == h.E_INVALID      # boundary kind
    assert lib.hmpcg_assemble(rho, C.byref(s), h.BC_DIRICHLET, 9, None) == h.E_INVALID     # face rule
    assert lib.hmpcg_assemble(None, C.byref(s), h.BC_DIRICHLET, h.FACE_INV_RHO, None) == h.E_INVALID
    assert lib.hmpcg_assemble(rho, None, h.BC_DIRICHLET, h.FACE_INV_RHO, None) == h.E_INVALID
    bad = h.SystemStruct()
    C.memmove(C.byref(bad), C.byref(s), C.sizeof(s))
    bad.dims[0] = 30
    assert lib.hmpcg_assemble(rho, C.byref(bad), h.BC_DIRICHLET, h.FACE_INV_RHO, None) == h.E_SHAPE
    bad.diag = None
    assert lib.hmpcg_assemble(rho, C.byref(bad), h.BC_DIRICHLET, h.FACE_INV_RHO, None) == h.E_INVALID
    assert lib.hmpcg_spmv(None, rho, rho, None) == h.E_INVALID
    assert lib.hmpcg_spmv(C.byref(s), None, rho, None) == h.E_INVALID


def test_other_entry_points_reject_null_handles():
    lib = h.lib()
    p = C.c_void_p(FAKE_BASE)
    s = h.SystemStruct()
    assert lib.hmpcg_infer_factors(None, C.byref(s), 1, p, h.BF16, None, None) == h.E_INVALID
    assert lib.hmpcg_train_step(None, C.byref(s), 1, 16, 3e-4, 1, None, None) == h.E_INVALID
    assert lib.hmpcg_get_weights(None, p, 10) == h.E_INVALID
    assert lib.hmpcg_get_grads(None, p, 10) == h.E_INVALID
    assert lib.hmpcg_apply_noalloc(None, p, p, None) == h.E_INVALID
    # GEMM: negative sizes and an unknown activation are refused
    assert lib.hmpcg_gemm_bf16(p, p, p, -1, 128, 128, None, 0, None) == h.E_INVALID
    assert lib.hmpcg_gemm_bf16(p, p, p, 128, 128, 128, None, 2, None) == h.E_INVALID


def test_status_strings_are_distinct():
    codes = [h.OK, h.NOT_CONVERGED, h.E_INVALID, h.E_SHAPE, h.E_CUDA, h.E_BREAKDOWN, h.E_NAN, h.E_TIMEOUT,
             h.E_NOMEM]
    texts = [h.status_string(c) for c in codes]
    assert len(set(texts)) == len(codes)
    assert all("unknown" not in t for t in texts)
    assert "unknown" in h.status_string(42)


C_PROGRAM = r"""
#include <stdio.h>
#include "hmpcg.h"
int main(void) {
  int32_t dims[3] = {32, 16, 16};
  hmpcg_system sys;
  hmpcg_config cfg = {0};
  cfg.max_n = 8192; cfg.max_batch = 1; cfg.max_nrhs = 1; cfg.leaf = 64; cfg.rank = 16;
  cfg.d_model = 128; cfg.n_layers = 4; cfg.n_heads = 4; cfg.d_mlp = 512;
  printf("%lld %lld %lld %d %s\n",
         (long long)hmpcg_packed_width(8192, 64, 16, HMPCG_PRE_LEARNED),
         (long long)hmpcg_system_bytes(3, dims),
         (long long)hmpcg_weight_count(&cfg),
         hmpcg_system_layout(3, dims, (void*)(uintptr_t)4096, &sys),
         hmpcg_status_string(HMPCG_E_BREAKDOWN));
  return (int)(sys.n != 8192);
}
"""


def test_header_is_plain_c_and_the_library_links_from_c(tmp_path):
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    import os
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    libdir = os.path.dirname(h.LIB_PATH)
    include = os.path.join(os.path.dirname(libdir), "include")
    exe = tmp_path / "abi"
    cc = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", include, str(src),
                         "-L", libdir, "-lhmpcg", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                        capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stderr
    width, nbytes, nweights, rc, text = run.stdout.split(" ", 4)
    assert int(width) == h.packed_width(8192, 64, 16, h.PRE_LEARNED)
    assert int(nbytes) == h.lib().hmpcg_system_bytes(3, _dims((32, 16, 16)))
    assert int(nweights) == sum(math.prod(s) for _, s in inputs.network_layout())
    assert int(rc) == h.OK and "breakdown" in text.lower()


def test_selftest_wait_rejects_bad_arguments_before_any_device_work():
    lib = h.lib()
    p = C.c_void_p(FAKE_BASE)
    assert lib.hmpcg_selftest_wait(None, p, 16, None) == h.E_INVALID
    assert lib.hmpcg_selftest_wait(p, None, 16, None) == h.E_INVALID
    assert lib.hmpcg_selftest_wait(p, p, 0, None) == h.E_INVALID                # at least one poll
    assert lib.hmpcg_selftest_wait(p, p, (1 << 24) + 1, None) == h.E_INVALID    # bounded by 2^24
    assert lib.hmpcg_selftest_wait(C.c_void_p(FAKE_BASE + 2), p, 16, None) == h.E_INVALID   # int32 alignment
