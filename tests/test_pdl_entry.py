"""Every kernel launched with programmatic stream serialisation waits for its predecessor.

A kernel launched through `pdl_launch` / `launch_pdl_bw` may be scheduled while the previous
kernel in its stream is still running; it must execute `pdl_entry()` (griddepcontrol.wait)
before it reads anything that kernel wrote.  A launch site added without the matching call in
the kernel would race silently, so this CPU test reads the CUDA sources and checks that the
body of every kernel passed to a programmatic launch helper calls pdl_entry() and does so
before its first global-memory access through a kernel argument (approximated: before the
first `[` index expression that is not a shared-memory declaration).
"""
import pathlib
import re

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2605_13343_gb300" / "csrc"
HELPERS = ("pdl_launch", "launch_pdl_bw", "launch_pdl")
# kernels that stage network weights into shared memory before the wait: no kernel of the
# forward writes weights, and the optimiser's kernels never trigger their dependents early
PRE_WAIT_WEIGHTS = {"encoder_mma_kernel", "fused_attn_kernel", "fused_ffn_kernel"}


def _sources():
    return {p.name: p.read_text() for p in sorted(CSRC.glob("*.cu*"))}


def _launched_kernels(srcs):
    names = {"gemm_bf16_tc_kernel"}   # launched by cudaLaunchKernelEx with the attribute in place
    pat = re.compile(r"\b(?:%s)\(\s*([A-Za-z_][A-Za-z_0-9]*)" % "|".join(HELPERS))
    for text in srcs.values():
        for m in pat.finditer(text):
            if m.group(1) != "void":   # the helpers' own definitions
                names.add(m.group(1))
    return names


def _kernel_body(srcs, name):
    pat = re.compile(r"__global__\s+void\s+(?:__launch_bounds__\((?:[^()]|\([^()]*\))*\)\s*)?" + re.escape(name) + r"\s*\(")
    for text in srcs.values():
        m = pat.search(text)
        if not m:
            continue
        i = text.index("{", m.end())
        depth, j = 0, i
        while True:
            if text[j] == "{":
                depth += 1
            elif text[j] == "}":
                depth -= 1
                if depth == 0:
                    return text[i + 1:j]
            j += 1
    return None


def test_programmatic_launches_wait_for_their_predecessor():
    srcs = _sources()
    names = _launched_kernels(srcs)
    assert len(names) > 20, names          # the helpers are found at all
    missing = []
    for name in sorted(names):
        body = _kernel_body(srcs, name)
        assert body is not None, f"no __global__ definition found for {name}"
        if "pdl_entry()" not in body:
            missing.append(name)
    assert not missing, f"launched with programmatic serialisation but never call pdl_entry(): {missing}"


def test_pdl_entry_comes_before_the_first_indexed_access():
    srcs = _sources()
    late = []
    for name in sorted(_launched_kernels(srcs)):
        body = _kernel_body(srcs, name)
        pos = body.index("pdl_entry()")
        head = body[:pos]
        # indexing before the wait is allowed only in shared-memory declarations and in
        # set-up that touches no kernel argument (TMEM allocation, barrier init)
        code = [ln for ln in head.splitlines()
                if "[" in ln and "__shared__" not in ln and "asm" not in ln and "mbar_init" not in ln
                and "smem_u32(" not in ln and not ln.strip().startswith("//")]
        if name in PRE_WAIT_WEIGHTS:
            continue
        reads = [ln for ln in code if re.search(r"\b(?:bar_full|bar_empty|acc_full|acc_empty|lgst|hwst|tile|red|pg|pb)\b", ln) is None]
        if reads:
            late.append((name, reads[:2]))
    assert not late, late
