"""Shared helpers of the GPU-vs-oracle parity tests (tolerances are stated here once).

Parity is per seed on identical Philox streams: the CUDA path (FP32 arithmetic, 64-bit
fixed-point tallies) and the FP64 oracle run the same packets.  Their difference is the FP32
rounding of each packet's deposits and positions (continuous, ~1e-6 of a packet's contribution)
plus the rare packet whose threshold/roulette or boundary decision flips under rounding.  Hence
(reading of the stated 1e-4 tolerance):

 (i)   per channel, sum_i |G - O| <= REL * sum_i A_i          (relative L1 over the field)
 (ii)  per pixel where the tally rests on many packets (A_i >= 1e-3 max A and
       sigma_i <= 3e-3 A_i, i.e. roughly >= 1e5 packet contributions):  |G - O| <= REL * A_i
 (iii) elsewhere |G - O| <= 3 sigma_i + REL * A_i

where A_i is the pixel's absolute tally (a_0 of the same packets with |W|; for forward runs
a_0 itself, since |a_n|, |b_n| <= a_0 per packet) and sigma_i the oracle's standard error of a_0.
The 1e-4 bound is stated for tallies of >= 1e6 packets: in a pixel visited by N packets, one
packet whose path diverged contributes ~1/N of the tally, so (ii) asks for N >~ 1e5.
"""
import numpy as np

REL = 1e-4


def f32(v):
    return float(np.float32(v))


def assert_parity(G, O, A, sigma, rel=REL, label="", unvisited_share=None, floor=0.0, outliers=None):
    """3D grazing paths: a path that runs within FP32 resolution of a voxel face, or through an
    edge, can cut through a neighbouring voxel on one side and not on the other, or for a
    different micro-length.  ``unvisited_share``: cells the oracle's packets never enter (A = 0,
    sigma = 0, where (iii) cannot apply) are held instead to sum |G| <= unvisited_share sum A;
    ``floor``: an absolute allowance added to (iii) for such micro-segments.  ``outliers`` =
    (fraction, share): on large sparse grids a packet whose FP32 and FP64 paths part can cross a
    cell that only one or two of the other side's packets touched; up to that fraction of the
    low-count cells may then exceed (iii) if together they carry at most that share of sum A."""
    G = np.asarray(G, np.float64)
    O = np.asarray(O, np.float64)
    A = np.abs(np.asarray(A, np.float64))
    assert G.shape == O.shape, (G.shape, O.shape)
    d = np.abs(G - O)
    tot = A.sum()
    for c in range(G.shape[0]):
        l1 = d[c].sum() / tot
        assert l1 <= rel, f"{label} channel {c}: relative L1 {l1:.3e} > {rel}"
    sigma = np.asarray(sigma, np.float64)
    hi = (A >= 1e-3 * A.max()) & (sigma <= 3e-3 * A)
    worst = float(np.max(d[:, hi] / A[hi])) if hi.any() else 0.0
    assert worst <= rel, f"{label}: per-pixel relative error {worst:.3e} > {rel}"
    lo = ~hi
    if unvisited_share is not None:
        zero = A == 0
        share = float(np.abs(G[:, zero]).sum(axis=1).max() / tot) if zero.any() else 0.0
        assert share <= unvisited_share, f"{label}: cells the oracle never enters carry {share:.3e} of the total"
        lo &= ~zero
    if lo.any():
        bound = 3 * sigma[lo] + rel * A[lo] + floor + 1e-30
        over = (d[:, lo] > bound).any(axis=0)
        if outliers is None:
            assert not over.any(), f"{label}: low-count pixels beyond 3 sigma"
        else:
            frac, share = outliers
            n_over = int(over.sum())
            excess = float(d[:, lo][:, over].sum(axis=1).max() / tot) if n_over else 0.0
            assert n_over <= frac * int(lo.sum()) and excess <= share, \
                f"{label}: {n_over} low-count cells beyond 3 sigma carrying {excess:.3e} of the total"
    return dict(max_rel=worst, l1=float(d.sum(axis=(1, 2)).max() / tot))
