"""Bounds of the unrolled sweeps' index maps, checked on the host.

These restate, index for index, the address arithmetic of the kernels in
paper_2209_11002_gb300/csrc/edaa_unrolled.cu (xw_part, xdot, dx_contract,
rank_record) and of edaa_unrolled_create's layout rules (padded X row stride
Ls, chunk-sum stride from xs_stride, RK and Lv), and check for shapes from the
smallest to the largest the engine takes (L <= 320, p <= 8) that every access
stays inside its buffer and every output entry is written exactly once.
No GPU needed."""
import itertools

import pytest

kT, kW, kMaxP, kLPMax = 256, 8, 8, 320 * 8
kXS = 4 * kMaxP * kT                      # Sm.xs floats
kDxPx, kDxB, kDxBlk, kKC = 8, 14, 96, 8   # dx_contract tiles and staging
SMS = 152


def padded_ls(L):                          # edaa_unrolled_create: resident X row stride
    Ls = (L + 3) & ~3
    return Ls + 4 if Ls % 8 == 0 else Ls


def xs_stride(L, P):                       # the host search for xw_part's quad stride
    Q, LP = (L + 3) >> 2, L * P
    C = min(8, max(1, kT // Q))
    best, bestw = Q, 1 << 30
    Qp = Q
    while Qp <= Q + 32 and C * 4 * P * Qp <= kXS:
        w = 1
        for c in range(C):
            for e0 in range(0, LP, 32):
                cnt = [0] * 32
                for lane in range(32):
                    e = e0 + lane
                    if e >= LP:
                        break
                    l, j = divmod(e, P)
                    b = (((c * 4 + (l & 3)) * P + j) * Qp + (l >> 2)) & 31
                    cnt[b] += 1
                    w = max(w, cnt[b])
        if w < bestw:
            best, bestw = Qp, w
        if bestw == 1:
            break
        Qp += 1
    return best


def cta_range(N, g, G=SMS):
    return N * g // G, N * (g + 1) // G


SHAPES = [(1, 100, 1), (23, 777, 3), (40, 1500, 4), (285, 13542, 4), (162, 94249, 6), (320, 20000, 8), (31, 999, 7)]


@pytest.mark.parametrize("L,N,P", SHAPES)
def test_xw_part_maps(L, N, P):
    Q, LP, Ls = (L + 3) >> 2, L * P, padded_ls(L)
    C, Qs = min(8, max(1, kT // Q)), xs_stride(L, P)
    assert Q * C <= kT and C * 4 * P * Qs <= kXS
    maxpx = (N + SMS - 1) // SMS + 1
    for g in (0, SMS // 2, SMS - 1):
        lo, hi = cta_range(N, g)
        npx = hi - lo
        assert npx <= maxpx
        written = set()
        for tid in range(Q * C):
            c, q = divmod(tid, Q)
            k0, k1 = lo + npx * c // C, lo + npx * (c + 1) // C
            assert lo <= k0 <= k1 <= hi
            if k1 > k0:  # X rows read: columns 4q..4q+3 of rows k0..k1-1 (row stride Ls)
                assert 4 * q + 3 < Ls and (k1 - 1 - lo) < maxpx
            for r, j in itertools.product(range(4), range(P)):
                idx = c * 4 * P * Qs + (r * P + j) * Qs + q
                assert 0 <= idx < kXS and idx not in written
                written.add(idx)
        for e in range(LP):          # the combine reads what the chunks wrote
            l, j = divmod(e, P)
            for c in range(C):
                assert ((c * 4 * P + (l & 3) * P + j) * Qs + (l >> 2)) in written


@pytest.mark.parametrize("L,N,P", SHAPES)
def test_xdot_maps(L, N, P):
    Ls, Qf = padded_ls(L), L >> 2
    outs = set()
    lo, hi = cta_range(N, SMS - 1)
    for warp in range(kW):
        for ib in range(lo + warp * 16, hi, kW * 16):
            for lane in range(32):
                h, pp = lane >> 3, lane & 7
                qa, qz = Qf * h // 4, Qf * (h + 1) // 4
                assert 0 <= qa <= qz <= Qf and 4 * qz <= L
                for i in (ib + pp, ib + 8 + pp):
                    if i < hi and h == 0:
                        for j in range(P):
                            assert (i, j) not in outs
                            outs.add((i, j))
            # every band read by exactly one quarter (the tail by quarter 3)
            bands = []
            for h in range(4):
                bands += list(range(4 * (Qf * h // 4), 4 * (Qf * (h + 1) // 4)))
            bands += list(range(4 * Qf, L))
            assert sorted(bands) == list(range(L)) and max(bands) < Ls
    assert outs == {(i, j) for i in range(lo, hi) for j in range(P)}


@pytest.mark.parametrize("L,N,P,T,K2", [(285, 13542, 4, 20, 5), (320, 20000, 8, 3, 2), (1, 100, 1, 1, 0), (40, 1500, 4, 3, 3)])
def test_dx_contract_and_rank_record_maps(L, N, P, T, K2):
    RK = (P * (1 + 2 * T * (K2 + 1)) + 7) & ~7
    Lv = (L + kDxB - 1) // kDxB * kDxB
    nbg = Lv // kDxB
    assert kKC * kDxBlk + kKC * Lv <= kXS          # staging fits Sm.xs
    assert (kKC * kDxBlk + kT - 1) // kT * kT >= kKC * kDxBlk
    assert (kKC * 322 + kT - 1) // kT * kT >= kKC * Lv
    # rank_record: the terms recorded fill columns 0..nr-1 of U and rows of V
    nr = P + T * (K2 * 2 * P + 2 * P)
    assert nr <= RK
    for nt in (1, 2):                               # V writes shared out among the CTAs
        LP, seen = L * P, set()
        for g in range(SMS):
            for tid in range(kT):
                e = g * kT + tid
                while e < nt * LP:
                    r, l = divmod(e, L)
                    t, j = divmod(r, P)
                    assert l < L <= Lv and t < nt and j < P and (r, l) not in seen
                    seen.add((r, l))
                    e += SMS * kT
        assert len(seen) == nt * LP
    # dx_contract: every (pixel, band) of a CTA written once, reads inside U, V, Us, Vs
    lo, hi = cta_range(N, 0)
    out = set()
    for p0 in range(lo, hi, kDxBlk):
        np_ = min(kDxBlk, hi - p0)
        ntile = (np_ + kDxPx - 1) // kDxPx * nbg
        for tau in range(ntile):
            pg, bg = divmod(tau, nbg)
            assert pg * kDxPx + kDxPx <= kDxBlk and bg * kDxB + kDxB <= Lv
            for q in range(kDxPx):
                i = pg * kDxPx + q
                if i < np_:
                    for b in range(kDxB):
                        l = bg * kDxB + b
                        if l < L:
                            assert (p0 + i, l) not in out
                            out.add((p0 + i, l))
    assert len(out) == (hi - lo) * L
