"""The tally-reduction ceiling probe (mc_reduction_probe) does exactly the additions it claims:
every word it may touch is one of the first C of a row, and the total is warps x iters x C."""
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
