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
