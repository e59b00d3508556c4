"""The measurement and test entry points of include/mcr_diag.h.

The tally-reduction probe (mc_reduction_probe) does exactly the additions it claims: every word it
may touch is one of the first C of a row, and the total is warps x iters x C.  The transport's
device Philox4x32-10 (mc_philox_blocks runs the very function the kernels call) reproduces the
generator's published known answers, and the transport's (packet, event) counter layout."""
import os

import pytest
import torch

from paper_1608_05238_gb300 import _build, mcr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    mcr.load()


@pytest.mark.parametrize("rows,row_words,C,iters,blocks,threads", [(1000, 80, 65, 50, 7, 96), (37, 12, 9, 333, 3, 64),
                                                                   (5, 144, 129, 10, 2, 1024)])
def test_probe_adds_one_per_coefficient_per_visit(rows, row_words, C, iters, blocks, threads):
    tally = torch.zeros(rows, row_words, dtype=torch.int64, device="cuda")
    mcr.reduction_probe(tally, C, iters, blocks, threads)
    torch.cuda.synchronize()
    t = tally.cpu()
    warps = blocks * threads // 32
    assert int(t.sum()) == warps * iters * C
    assert not t[:, C:].any()
    # within a row all C words were hit equally often (each visit adds 1 to every one of them)
    assert torch.equal(t[:, :C], t[:, :1].expand(-1, C))


def test_probe_rejects_bad_arguments():
    tally = torch.zeros(4, 8, dtype=torch.int64, device="cuda")
    with pytest.raises(mcr.McrError):
        mcr.reduction_probe(tally, 9, 1, 1, 32)   # C > row_words
    with pytest.raises(mcr.McrError):
        mcr.reduction_probe(tally, 8, 1, 1, 48)   # threads not a multiple of 32


def test_device_philox_known_answers():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [[int(x, 16) for x in line.split()] for line in open(path) if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    got = mcr.philox_blocks([r[0:4] for r in rows], [r[4:6] for r in rows])
    assert got == [tuple(r[6:10]) for r in rows]


def test_device_philox_counter_layout_matches_oracle():
    """Counter (packet_lo, packet_hi, event, 0), key (seed_lo, seed_hi ^ stream_id): the device
    blocks equal the oracle's for packet ids above 2^32 and several events."""
    oracle = pytest.importorskip("oracle")
    seed, stream_id = 0x0123456789ABCDEF, 7
    key = (seed & 0xFFFFFFFF, (seed >> 32) ^ stream_id)
    ctrs = [((p & 0xFFFFFFFF), p >> 32, e, 0) for p in (0, 1, 12345, (1 << 32) + 5) for e in (0, 1, 2, 1000)]
    got = mcr.philox_blocks(ctrs, [key] * len(ctrs))
    for c, g in zip(ctrs, got):
        assert g == tuple(int(v) for v in oracle.philox4x32_10(c, key))


def test_philox_hook_rejects_bad_arguments():
    with pytest.raises(ValueError):
        mcr.philox_blocks([], [])
