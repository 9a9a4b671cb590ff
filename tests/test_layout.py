"""Host packing of the device layout (no GPU needed): the chunking of the
component order and the per-chunk halo, checked through opf_chunk_stats.

Every local variable lives in exactly one chunk; in a chunk's halo each copy
of a global is either one of the chunk's own locals or a copy owned by
another chunk (an external copy), so copies - external = locals per chunk.
A single chunk has no boundary, and the neighbour relation is symmetric (two
chunks that share a global read each other's copies)."""
import numpy as np
import pytest

from paper_2501_08293_b300 import feeders as F
from paper_2501_08293_b300 import opf


@pytest.mark.parametrize("chunks", [1, 2, 4, 17, 40])
def test_chunk_layout_invariants_123bus(chunks):
    p = opf.Problem.from_feeder(F.feeder_123(1), upload=False, chunks=chunks)
    try:
        d = p.dims
        st = p.chunk_stats()
        assert d.n_blocks == chunks
        assert int(st["locals"].sum()) == d.n_local
        assert (st["locals"] > 0).all() and (st["tiles"] > 0).all()
        assert np.array_equal(st["copies"] - st["external_copies"], st["locals"])
        assert (st["halo"] >= st["boundary_halo"]).all() and (st["boundary_halo"] >= 0).all()
        assert (st["tiles"] >= st["interior_tiles"]).all()
        assert (st["max_warp_quads"] <= st["quads"] + 2 * st["tiles"]).all()
        if chunks == 1:
            assert int(st["boundary_halo"].sum()) == 0 and int(st["external_copies"].sum()) == 0
            assert int(st["neighbours"].sum()) == 0
        else:
            assert (st["neighbours"] >= 1).all()
            assert int(st["neighbours"].sum()) % 2 == 0
            # a boundary entry has at least one copy outside the chunk
            assert (st["external_copies"] >= st["boundary_halo"]).all()
    finally:
        p.close()


def test_default_chunking_of_the_8500_class_feeder():
    """296 work-balanced chunks (two per SM of a 148-SM part) for the
    8500-class feeder, each with a small boundary next to its interior."""
    p = opf.Problem.from_feeder(F.feeder_8500(1), upload=False)
    try:
        d = p.dims
        st = p.chunk_stats()
        assert d.n_blocks == 296
        assert int(st["locals"].sum()) == d.n_local
        assert np.array_equal(st["copies"] - st["external_copies"], st["locals"])
        # work balance: no chunk holds far more locals than the mean
        assert st["locals"].max() <= 1.5 * st["locals"].mean()
        assert st["boundary_halo"].sum() < 0.25 * st["halo"].sum()
    finally:
        p.close()
