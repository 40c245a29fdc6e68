"""Source checks of the CUDA kernels that need no GPU.

A warp-synchronous intrinsic with the full mask must be reached by every
lane of the warp; one placed in a short-circuit operand (`a && __shfl_sync(..)`)
or a conditional expression is skipped by some lanes and the warp waits
forever.  These checks keep such calls on lines of their own."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SYNC_INTRINSICS = r"__(shfl(_up|_down|_xor)?|all|any|ballot|reduce_\w+|match_\w+)_sync"


def kernel_sources():
    pat = os.path.join(ROOT, "paper_2106_14402_gb300", "csrc*", "*")
    return [p for p in glob.glob(pat) if p.endswith((".cu", ".cuh"))]


def test_no_warp_sync_call_behind_short_circuit():
    bad = []
    for path in kernel_sources():
        for n, line in enumerate(open(path), 1):
            code = line.split("//")[0]
            m = re.search(SYNC_INTRINSICS, code)
            if not m:
                continue
            before = code[:m.start()]
            if "&&" in before or "||" in before or re.search(r"\?[^:]*$", before):
                bad.append(f"{os.path.basename(path)}:{n}: {line.strip()}")
    assert not bad, "\n".join(bad)
