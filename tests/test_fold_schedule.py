"""The folded preconditioner's persistent-launch work list, checked on the host (no GPU).

The launch runs the four folded products of the Laplacian solve (Sec. 3.3, the DCT eigenbasis
products folded into even / odd halves) as one list of tiles; pair p takes items p, p + P, ...
in order, and a tile waits on counters that the tiles producing its input rows complete.  The
list comes from the library's own builder (irls_debug_fold_schedule, the same code the launch's
set-up runs).  The checks restate, from the fold's algebra, which rows each stage reads and
writes, and need nothing from the builder but its output:

- every output tile of every product is computed exactly once (half-width splits included);
- every counter a tile waits for is completed by exactly the tiles that write the rows it reads,
  and the count it waits for is what those tiles add (one per CTA of the pair);
- every producer precedes its consumers in the list, and the static pair assignment runs to the
  end (no deadlock) when every pair is resident;
- the r^T z flags of stage 2 mark each pair's last tile of the image's run.
"""
import os

import numpy as np
import pytest

import synthetic

F = {n: i for i, n in enumerate(
    ["stage", "image", "local", "m0", "n0", "width", "nkb", "dual", "half", "sig", "ndep"] +
    [f"dep{d}" for d in range(8)] + [f"need{d}" for d in range(8)] +
    ["rho_end", "rho_nslot", "M", "N", "K", "prob"])}
PROBS_PER_IMAGE = (2, 4, 2, 1)


@pytest.fixture(scope="module")
def B():
    from paper_2401_09961_gb300 import _binding
    if not os.path.exists(_binding.LIB_PATH):
        from paper_2401_09961_gb300 import build
        build.build()
    _binding.lib()
    assert _binding.FOLD_SCHED_INTS == len(F)
    return _binding


def rup(x, m):
    return (x + m - 1) // m * m


def dims(H, W):
    """Padded half sides of the fold: (n + 1) / 2 rounded up to 256, and H rounded up to 256."""
    hNp, hMp = rup((H + 1) // 2, 256), rup((W + 1) // 2, 256)
    return hNp, hMp, rup(H, 256)


def expected_problems(H, W):
    """(M, N, K) of each stage's products for one image, restated from the fold:
    stage 0 folds R along j and multiplies by the half bases of side W (hMp x hNp outputs),
    stage 1 multiplies by the half bases of side H and divides by the eigenvalue sums,
    stage 2 unfolds along i (two operand sets), stage 3 unfolds along j into Z (H x W)."""
    hNp, hMp, Hp = dims(H, W)
    return [(hMp, hNp, hMp), (hMp, hNp, hNp), (hNp, hMp, hNp), (Hp, hMp, hMp)]


def schedule(B, shapes, pairs):
    rec, n_ctr, cap = B.fold_schedule(shapes, pairs)
    return rec, n_ctr, cap


def col(rec, name):
    return rec[:, F[name]]


def check_schedule(rec, n_ctr, cap, shapes, pairs):
    n = len(rec)
    T = len(shapes)
    assert 0 < n <= cap
    # ---- problems: dimensions, and every output tile exactly once
    for t, (H, W) in enumerate(shapes):
        exp = expected_problems(H, W)
        for k in range(4):
            for q in range(PROBS_PER_IMAGE[k]):
                prob = PROBS_PER_IMAGE[k] * t + q
                sel = rec[(col(rec, "stage") == k) & (col(rec, "prob") == prob)]
                assert len(sel) > 0
                assert (sel[:, F["image"]] == t).all()
                M, N, K = exp[k]
                assert (sel[:, [F["M"], F["N"], F["K"]]] == [M, N, K]).all(), (t, k, q)
                assert (sel[:, F["nkb"]] == K // 64).all()
                assert (sel[:, F["dual"]] == (1 if k >= 2 else 0)).all()
                cover = np.zeros((M // 256, N), dtype=np.int32)
                for r in sel:
                    assert r[F["m0"]] % 256 == 0 and r[F["n0"]] % 128 == 0
                    cover[r[F["m0"]] // 256, r[F["n0"]]:r[F["n0"]] + r[F["width"]]] += 1
                assert (cover == 1).all(), (t, k, q)
    # ---- which counter holds which rows: the producing tiles' row panels
    producers = {}
    for i in range(n):
        c = rec[i, F["sig"]]
        if c >= 0:
            producers.setdefault(int(c), []).append(i)
    assert sorted(producers) == list(range(n_ctr))
    panel = {}   # counter -> (image, stage, problem, row block)
    for c, items in producers.items():
        keys = {(int(rec[i, F["image"]]), int(rec[i, F["stage"]]), int(rec[i, F["prob"]]),
                 int(rec[i, F["m0"]]) // 256) for i in items}
        assert len(keys) == 1, c          # one counter, one row panel of one product
        panel[c] = keys.pop()
        # all tiles of that panel signal it (full panels only)
        img, k, prob, b = panel[c]
        sel = np.where((col(rec, "stage") == k) & (col(rec, "prob") == prob) &
                       (col(rec, "m0") // 256 == b))[0]
        assert sorted(sel.tolist()) == sorted(items)
    assert not (col(rec, "sig")[col(rec, "stage") == 3] >= 0).any()   # Z has no consumers
    # ---- what each tile must wait for, restated
    for i in range(n):
        k, t = int(rec[i, F["stage"]]), int(rec[i, F["image"]])
        H, W = shapes[t]
        hN = (H + 1) // 2
        q = int(rec[i, F["prob"]]) - PROBS_PER_IMAGE[k] * t
        m0, n0 = int(rec[i, F["m0"]]), int(rec[i, F["n0"]])
        if k == 0:
            want = set()                                  # reads the folded residual
        elif k == 1:
            x = q >> 1                                    # A = T1 of parity x, rows m0 .. + 256
            want = {(t, 0, 2 * t + x, m0 // 256)}
        elif k == 2:
            x = q                                         # B = T2(x, e) and T2(x, o), rows n0 ..
            want = {(t, 1, 4 * t + 2 * x + y, n0 // 256) for y in (0, 1)}
        else:                                             # A = rows r of T3e, T3o: stage-3 row
            rows = range(m0, min(m0 + 256, H))            # i' = r (r < hN) or H - 1 - r
            blocks = {(r if r < hN else H - 1 - r) // 256 for r in rows}
            want = {(t, 2, 2 * t + x, b) for x in (0, 1) for b in blocks}
        nd = int(rec[i, F["ndep"]])
        deps = [int(rec[i, F[f"dep{d}"]]) for d in range(nd)]
        needs = [int(rec[i, F[f"need{d}"]]) for d in range(nd)]
        assert len(set(deps)) == nd
        assert {panel[c] for c in deps} == want, (i, k)
        for c, need in zip(deps, needs):
            assert need == 2 * len(producers[c])         # each CTA of a pair adds one
            assert max(producers[c]) < i                  # producers first in the list
    # ---- r^T z flags: each image's stage-2 tiles are one run; each pair's last tile ends it
    for t in range(T):
        run = np.where((col(rec, "stage") == 1) & (col(rec, "image") == t))[0]
        a, b = run[0], run[-1] + 1
        assert (run == np.arange(a, b)).all()
        assert (rec[a:b, F["rho_nslot"]] == 2 * min(pairs, b - a)).all()
        for p in range(pairs):
            mine = [j for j in range(a, b) if j % pairs == p]
            if mine:
                assert rec[mine[-1], F["rho_end"]] == 1
                assert (rec[mine[:-1], F["rho_end"]] == 0).all()
    # ---- half-width splits: stage-3 tiles at the end of the list, in consecutive halves
    halves = np.where(col(rec, "half") == 1)[0]
    assert len(halves) % 2 == 0
    if len(halves):
        assert halves[0] == n - len(halves) and (col(rec, "stage")[halves] == 3).all()
        assert len(halves) // 2 <= min(pairs, 1024)
        for j in range(halves[0], n, 2):
            a, b = rec[j], rec[j + 1]
            assert a[F["prob"]] == b[F["prob"]] and a[F["local"]] == b[F["local"]]
            assert a[F["m0"]] == b[F["m0"]] and b[F["n0"]] == a[F["n0"]] + 128
    # ---- the static assignment runs to the end with all pairs resident
    count = np.zeros(n_ctr, dtype=np.int64)
    nxt = list(range(min(pairs, n)))
    done = 0
    while True:
        progressed = False
        for p in range(len(nxt)):
            i = nxt[p]
            if i >= n:
                continue
            nd = int(rec[i, F["ndep"]])
            if all(count[rec[i, F[f"dep{d}"]]] >= rec[i, F[f"need{d}"]] for d in range(nd)):
                if rec[i, F["sig"]] >= 0:
                    count[rec[i, F["sig"]]] += 2
                nxt[p] = i + pairs
                done += 1
                progressed = True
        if not progressed:
            break
    assert done == n, f"deadlock after {done} of {n} items"


@pytest.mark.parametrize("shape", [(256, 256), (4096, 4096), (257, 1025), (511, 769),
                                   (1024, 2048), (4000, 2000)])
@pytest.mark.parametrize("pairs", [1, 3, 76])
def test_single_image_schedule(B, shape, pairs):
    rec, n_ctr, cap = schedule(B, [shape], pairs)
    check_schedule(rec, n_ctr, cap, [shape], pairs)


@pytest.mark.parametrize("pairs", [2, 76])
def test_batched_schedule_of_uneven_tiles(B, pairs):
    shapes = synthetic.batched_tile_shapes(n=64, seed_base=1000)
    rec, n_ctr, cap = schedule(B, shapes, pairs)
    check_schedule(rec, n_ctr, cap, shapes, pairs)


def test_large_non_square_schedule(B):
    shapes = [(4000, 16000)]
    rec, n_ctr, cap = schedule(B, shapes, 76)
    check_schedule(rec, n_ctr, cap, shapes, 76)


def test_half_width_split_only_where_it_pays(B):
    # one pair: a split adds work and cannot fill an idle pair
    rec, _, _ = schedule(B, [(4096, 4096)], 1)
    assert not col(rec, "half").any()
    # 76 pairs at 4096 x 4096: 128 stage-3 tiles fill 1.7 waves; the tail is split
    rec, _, _ = schedule(B, [(4096, 4096)], 76)
    assert col(rec, "half").sum() > 0


def test_argument_checks(B):
    import ctypes
    L = B.lib()
    H = (ctypes.c_int * 1)(255)
    W = (ctypes.c_int * 1)(512)
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    args = (ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    assert L.irls_debug_fold_schedule(1, H, W, 4, *args, None, 0) == -2
    H[0] = 512
    assert L.irls_debug_fold_schedule(1, H, W, 0, *args, None, 0) == -1
    assert L.irls_debug_fold_schedule(0, H, W, 4, *args, None, 0) == -1
    assert L.irls_debug_fold_schedule(1, None, W, 4, *args, None, 0) == -1
    assert L.irls_debug_fold_schedule(1, H, W, 4, *args, None, 0) == 0
    buf = (ctypes.c_int * 33)()
    assert L.irls_debug_fold_schedule(1, H, W, 4, *args, buf, 1) == -1   # too small
    assert a.value > 1


def test_checker_catches_planted_mistakes(B):
    """Each plausible builder mistake, planted in a copy of the record, fails a check."""
    shape, pairs = [(1000, 1536)], 5      # H = 1000: stage-3 tiles that straddle the fold line
    rec, n_ctr, cap = schedule(B, shape, pairs)
    check_schedule(rec, n_ctr, cap, shape, pairs)
    stage = col(rec, "stage")

    def fails(mutate):
        r = rec.copy()
        mutate(r)
        with pytest.raises(AssertionError):
            check_schedule(r, n_ctr, cap, shape, pairs)

    i1 = int(np.where(stage == 1)[0][3])
    i3 = int(np.where((stage == 3) & (col(rec, "ndep") > 2))[0][0])
    i2 = int(np.where(stage == 2)[0][0])

    def need_off_by_one(r):       # a wait for one count more than the panel reaches
        r[i1, F["need0"]] += 1
    fails(need_off_by_one)

    def dep_dropped(r):           # a stage-3 tile that misses one T3 panel it reads
        r[i3, F["ndep"]] -= 1
    fails(dep_dropped)

    def wrong_panel(r):           # stage-2 tile waits on the wrong T2 row panel
        r[i2, F["dep0"]] = r[i2, F["dep1"]]
    fails(wrong_panel)

    def consumer_first(r):        # a consumer placed before its producers
        r[[0, i1]] = r[[i1, 0]]
    fails(consumer_first)

    def tile_twice(r):            # one output tile computed twice, another never
        r[i2, F["n0"]] = (r[i2, F["n0"]] + 256) % r[i2, F["N"]]
    fails(tile_twice)

    def rho_flag(r):              # r^T z run end on the wrong tile of a pair
        j = int(np.where((stage == 1) & (col(rec, "rho_end") == 1))[0][0])
        r[j, F["rho_end"]] = 0
        r[j - pairs, F["rho_end"]] = 1
    fails(rho_flag)
