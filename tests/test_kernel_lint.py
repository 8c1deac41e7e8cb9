"""Static guard for the CUDA sources: a warp-synchronous intrinsic (shuffle, ballot, syncwarp,
match) must never be the right operand of &&, || or ?:, where short-circuit evaluation would let
some lanes skip it (divergent warp-synchronous instructions are undefined behaviour)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_14294_b300", "csrc")
SYNC = re.compile(r"(&&|\|\||\?)[^;{}]*__(shfl\w*|ballot_sync|syncwarp|any_sync|all_sync|match\w*)\s*\(")


def test_no_short_circuited_warp_sync():
    bad = []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith(".cu"):
            continue
        for i, line in enumerate(open(os.path.join(CSRC, f)), 1):
            code = line.split("//")[0]
            if SYNC.search(code):
                bad.append(f"{f}:{i}: {line.strip()}")
    assert not bad, "\n".join(bad)


TRAP = re.compile(r"__trap\s*\(|\bassert\s*\(|\btrap;|\bbrkpt\b")


def test_no_deliberate_faults_in_the_cuda_sources():
    """Failure paths report through status words the host reads (time limits, overflow flags),
    never by stopping the device: no trap, breakpoint or device-side assert anywhere."""
    bad = []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith((".cu", ".h", ".cpp")):
            continue
        for i, line in enumerate(open(os.path.join(CSRC, f)), 1):
            if TRAP.search(line.split("//")[0]):
                bad.append(f"{f}:{i}: {line.strip()}")
    assert not bad, "\n".join(bad)
