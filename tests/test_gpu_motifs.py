"""Motif census on the GPU (one batched launch per motif size) against the oracle's census by
definition and the oracle's non-induced counts."""
import pytest

import inputs
import oracle
from paper_2103_14294_b300 import motifs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [3, 4, 5])
def test_census_matches_oracle(gpu_lib, k):
    huge = gpu_lib
    for g in (inputs.gnp(22, 1, 4, 31), inputs.rmat(5, 4, 9)):
        G = huge.Graph(g.offsets, g.adj)
        rows = motifs.census(G, k)
        assert len(rows) == len(motifs.patterns(k))
        for p, nonind, _ in rows:
            assert nonind == oracle.count(g, k, p, oracle.symmetry_breaking_order(k, p)), p
        got = {oracle.motif_key(k, p): ind for p, _, ind in rows if ind}
        assert got == oracle.motif_census(g, k)
