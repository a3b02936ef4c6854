"""Index identities the CUDA kernels rely on, checked exhaustively on the CPU.

* the line FFT's register layouts: element t + T c of thread t, register c; after the forward
  transform frequency b(t) + K c with b(t) = t, or at P = 4096 (the group-local last exchange)
  b(t) = (t >> 4) + 16 (t & 15);
* the half chirp table (entry f for f <= P/2, P - f above; padded i + i/16 at P = 4096) read
  at two per-thread offsets with one constant step per register;
* the n = P/2 forms: the crop rows or columns P/4 .. 3P/4 are exactly the registers 4 .. 11;
* the middle-half forms: a box inside P/4 .. 3P/4 touches only the registers 4 .. 11;
* the split of pass B's partial last round of column groups: every (group, plane) item goes
  to exactly one block, every block's slots stay below tslots, and the combine step visits
  every block that holds a part of its group.
"""

import pytest


def spad(a):
    return a + (a >> 4)


def layout(P):
    T = P // 16
    hw = P == 4096
    def fpos(t, c):
        return ((t >> 4) + (T // 16) * (t & 15) + T * c) if hw else t + T * c
    return T, hw, fpos


POW2 = [1 << k for k in range(4, 13)]


@pytest.mark.parametrize("P", POW2)
def test_chirp_offsets_equal_the_folded_half_table(P):
    T, hw, fpos = layout(P)
    K = T + T // 16 if hw else T
    for t in range(T):
        b = fpos(t, 0)
        assert 0 <= b < T
        lo = spad(b) if hw else b
        hi = spad(T - b) if hw else T - b
        for c in range(16):
            f = fpos(t, c)
            i = f if f <= P // 2 else P - f
            want = spad(i) if hw else i
            got = lo + K * c if c < 8 else hi + K * (15 - c)
            assert got == want, (P, t, c)


@pytest.mark.parametrize("P", [1024, 2048, 4096])
def test_half_form_crop_is_registers_4_to_11(P):
    T, _, _ = layout(P)
    n, lo = P // 2, P // 4
    for t in range(T):
        crop = {c for c in range(16) if 0 <= t + T * c - lo < n}
        assert crop == set(range(4, 12))


@pytest.mark.parametrize("P", [1024, 2048, 4096])
def test_middle_half_box_is_inside_registers_4_to_11(P):
    T, _, _ = layout(P)
    w3 = 1140 * P // 4096                      # the distance-3 box of the large workload
    for x0, w in [(P // 4, P // 2), (P // 4 + 3, 100), (P // 2 - w3 // 2, w3),
                  (3 * P // 4 - 1, 1)]:
        assert P // 4 <= x0 and x0 + w <= 3 * P // 4
        for t in range(T):
            for c in range(16):
                if x0 <= t + T * c < x0 + w:
                    assert 4 <= c < 12


def split_plan(ngroups, nblk, per):
    """Pass B's split of a partial last round (pb_split 2): whole groups for the full rounds,
    the last round's (group, plane) items dealt evenly; returns {block: [(group, q0, q1,
    slot)]}, tslots."""
    rounds = ngroups // nblk
    tail = ngroups - rounds * nblk
    titems = tail * per
    rng = (titems + nblk - 1) // nblk
    tslots = (rng + per - 1) // per + 1 if titems else 0
    plan = {}
    for bid in range(nblk):
        ti0, ti1 = titems * bid // nblk, titems * (bid + 1) // nblk
        segs = []
        sg = rounds
        while True:
            tg = ti0 // per + (sg - rounds)
            g0 = tg * per
            if ti0 >= ti1 or g0 >= ti1:
                break
            q0 = ti0 - g0 if ti0 > g0 else 0
            q1 = ti1 - g0 if ti1 - g0 < per else per
            segs.append((rounds * nblk + tg, q0, q1, sg - rounds))
            sg += 1
        plan[bid] = segs
    return plan, tslots, rounds, tail


@pytest.mark.parametrize("ngroups,nblk,per", [
    (1024, 152, 240), (1024, 152, 16), (1024, 152, 8), (913, 152, 2), (128, 152, 720),
    (256, 304, 180), (1000, 7, 3), (30, 29, 1), (64, 60, 5)])
def test_last_round_split_covers_every_item_once(ngroups, nblk, per):
    plan, tslots, rounds, tail = split_plan(ngroups, nblk, per)
    seen = {}
    for bid, segs in plan.items():
        for grp, q0, q1, slot in segs:
            assert rounds * nblk <= grp < ngroups and 0 <= q0 < q1 <= per
            assert 0 <= slot < tslots
            for q in range(q0, q1):
                assert (grp, q) not in seen
                seen[(grp, q)] = bid
    assert len(seen) == tail * per
    # the combine step of group tg looks at blocks blo .. bhi (as k_pass_b_tail does) and takes
    # slot tg - i0 / per of each block whose range meets the group
    titems = tail * per
    for tg in range(tail):
        g0, g1 = tg * per, (tg + 1) * per
        blo = max(0, g0 * nblk // titems - 1)
        bhi = min(nblk - 1, g1 * nblk // titems + 1)
        holders = {bid for (grp, _), bid in seen.items() if grp == rounds * nblk + tg}
        assert holders <= set(range(blo, bhi + 1))
        for bid in holders:
            i0 = titems * bid // nblk
            slot = tg - i0 // per
            assert any(s[0] == rounds * nblk + tg and s[3] == slot for s in plan[bid])


def test_host_call_parts_partition_every_chunk():
    """holo_gradient_host's split of a chunk into parts (weights of the first `parts` entries,
    rounded prefix sums): consecutive, non-empty parts covering [0, nk) for every nk up to
    2000, with the constants read from the library source."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2407_20304_gb300", "csrc", "holo_api.cu")).read()
    n_parts = int(re.search(r"constexpr int kHostParts = (\d+);", src).group(1))
    min_part = int(re.search(r"constexpr int kHostMinPart = (\d+);", src).group(1))
    weights = [int(x) for x in re.search(r"kHostWeights\[kHostParts\] = \{([^}]*)\}", src)
               .group(1).split(",")]
    assert len(weights) == n_parts
    for nk in range(1, 2001):
        parts = min(n_parts, nk // min_part) if nk >= 2 * min_part else 1
        if parts == 1:
            continue
        wsum = sum(weights[:parts])
        bound = [(nk * sum(weights[:p]) + wsum // 2) // wsum for p in range(parts)] + [nk]
        assert bound[0] == 0 and bound[-1] == nk
        assert all(bound[p + 1] > bound[p] for p in range(parts)), nk
