"""GPU path vs the FP64 oracle, through the C ABI.

Acceptance (per the method: pruning never changes a decision of the standard
variant):
  * labels bit-exact, except points whose FP64 top-2 similarity gap is below
    1e-6 (there the FP32 similarities may legitimately order differently);
  * centers within 1e-5 (L2 per center; centers are unit vectors) and the
    objective J within 1e-5 relative;
  * the GPU variants agree with each other bit for bit (one canonical FP32
    similarity everywhere).
Checks are teacher-forced per step: the oracle assigns with the GPU's centers
and updates with the GPU's labels, so one near-tie cannot derail the rest.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2107_04074_gb300 import skm  # noqa: E402

GAP = 1e-6
CTOL = 1e-5
VARIANTS = ["standard", "hamerly", "elkan", "simp_hamerly", "simp_elkan", "yinyang"]


def _dev(csr):
    return (torch.from_numpy(csr.row_ptr).cuda(), torch.from_numpy(csr.col).cuda(),
            torch.from_numpy(csr.val).cuda())


def _km(csr, k, variant, init, dev=None, **kw):
    rp, col, val = dev if dev is not None else _dev(csr)
    return skm.KMeans(csr.n, csr.d, rp, col, val, k, variant=variant, init_rows=init, **kw)


def _check_assign(X, ri, C_used, prev, got, rows=None):
    """Oracle assignment with the GPU's centers; returns #labels compared."""
    if rows is not None:
        sub = X_rows(X, rows)
        lab, _, _, _, gap = oracle.assign(sub, oracle.rinv(sub), C_used.astype(np.float64), prev[rows])
        got = got[rows]
    else:
        lab, _, _, _, gap = oracle.assign(X, ri, C_used.astype(np.float64), prev)
    ok = (lab == got) | (gap < GAP)
    bad = np.flatnonzero(~ok)
    assert bad.size == 0, f"{bad.size} label mismatches, e.g. rows {bad[:5]}"
    return int(np.sum(gap >= GAP))


_CSR_CACHE = {}


def X_rows(X, rows):
    key = id(X)
    csr = _CSR_CACHE[key]
    return oracle.Data.from_csr(csr.rows(rows))


def _teacher_forced(csr, k, variant, init, iters, sample=None, seed=0):
    X = oracle.Data.from_csr(csr)
    _CSR_CACHE[id(X)] = csr
    ri = oracle.rinv(X)
    km = _km(csr, k, variant, init)
    prev = np.full(csr.n, -1, dtype=np.int32)
    rng = np.random.default_rng(seed)
    seq = []
    for it in range(iters):
        C = km.centers()
        ch = km.assign()
        lab = km.labels()
        assert ch == int(np.sum(lab != prev))
        rows = None if sample is None else np.sort(rng.choice(csr.n, size=min(sample, csr.n), replace=False))
        _check_assign(X, ri, C, prev, lab, rows)
        seq.append(lab.copy())
        if ch == 0:
            break
        J = km.update_centers()
        Cn = km.centers()
        Co, _, Jo = oracle.update(X, ri, lab, C.astype(np.float64))
        assert np.max(np.linalg.norm(Cn - Co, axis=1)) < CTOL
        assert abs(J - Jo) <= CTOL * abs(Jo)
        prev = lab
    km.close()
    return seq


@pytest.fixture(scope="module")
def tiny():
    return synth.tfidf(synth.CSR_TINY)


@pytest.fixture(scope="module")
def mid():
    # the RCV-1-like recipe at 20k rows: several SpMM tiles, ragged rows
    return synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=20000, d=20000, seed=12))


@pytest.mark.parametrize("variant", VARIANTS)
def test_tiny_teacher_forced(tiny, variant):
    init = synth.init_rows(tiny.n, 20, 1)
    _teacher_forced(tiny, 20, variant, init, 20)


@pytest.mark.parametrize("variant", VARIANTS)
def test_mid_teacher_forced(mid, variant):
    init = synth.init_rows(mid.n, 100, 2)
    _teacher_forced(mid, 100, variant, init, 12, sample=3000)


def test_variants_bit_identical_and_match_oracle_trajectory(tiny):
    """All GPU variants give the same label sequence, equal to the oracle's
    full (untouched) trajectory wherever no near-tie occurred."""
    init = synth.init_rows(tiny.n, 20, 1)
    X = oracle.Data.from_csr(tiny)
    tr = oracle.run(X, oracle.unit_rows(X, init), "standard", max_iters=20)
    dev = _dev(tiny)
    seqs = {}
    for v in VARIANTS:
        km = _km(tiny, 20, v, init, dev)
        labs, Js = [], []
        for _ in range(20):
            ch = km.assign()
            labs.append(km.labels())
            if ch == 0:
                break
            Js.append(km.update_centers())
        seqs[v] = (labs, Js)
        km.close()
    ref = seqs["standard"][0]
    for v, (labs, Js) in seqs.items():
        assert len(labs) == len(ref), v
        for a, b in zip(labs, ref):
            np.testing.assert_array_equal(a, b)
    assert len(ref) == tr.iters
    for t in range(tr.iters):
        np.testing.assert_array_equal(ref[t], tr.labels[t])
    np.testing.assert_allclose(seqs["standard"][1], tr.J[:len(seqs["standard"][1])], rtol=CTOL)


@pytest.mark.parametrize("variant", ["hamerly", "elkan", "simp_hamerly", "simp_elkan", "yinyang"])
def test_bounds_hold_against_exact_similarities(mid, variant):
    """Section 4 invariants after every assignment: l(i) <= <x,c_a>,
    u(i,j) >= <x,c_j> (Elkan), u(i) >= max_{j != a} <x,c_j> (Hamerly),
    u(i,G) >= max_{j in G, j != a} <x,c_j> (Yin-Yang, groups of 8)."""
    k = 100
    init = synth.init_rows(mid.n, k, 3)
    X = oracle.Data.from_csr(mid)
    ri = oracle.rinv(X)
    Xd = None
    km = _km(mid, k, variant, init)
    rows = np.random.default_rng(5).choice(mid.n, 1500, replace=False)
    sub = mid.rows(rows)
    Xs = sub.dense() * oracle.rinv(oracle.Data.from_csr(sub))[:, None]
    for it in range(8):
        km.assign()
        C = km.centers().astype(np.float64)
        l, u = km.bounds()
        lab = km.labels()
        S = Xs @ C.T
        s_a = S[np.arange(len(rows)), lab[rows]]
        assert np.all(l[rows] <= s_a + 1e-12)
        if variant == "yinyang":
            S2 = S.copy()
            S2[np.arange(len(rows)), lab[rows]] = -np.inf
            for g in range(u.shape[0]):
                m = S2[:, 8 * g:8 * g + 8].max(axis=1)
                assert np.all(u[g, rows] >= m - 1e-12)
        elif u.ndim == 2:
            uu = u[rows]
            mask = np.ones_like(S, dtype=bool)
            mask[np.arange(len(rows)), lab[rows]] = False
            assert np.all(uu[mask] >= S[mask] - 1e-12)
        else:
            S2 = S.copy()
            S2[np.arange(len(rows)), lab[rows]] = -np.inf
            assert np.all(u[rows] >= S2.max(axis=1) - 1e-12)
        km.update_centers()
    km.close()
    del Xd, ri


def test_pruning_saves_similarities(mid):
    init = synth.init_rows(mid.n, 100, 2)
    dev = _dev(mid)
    tot = {}
    for v in ["standard", "hamerly", "elkan", "yinyang"]:
        km = _km(mid, 100, v, init, dev)
        s = 0
        for _ in range(15):
            ch = km.assign()
            s += km.stats().last_sims
            if ch == 0:
                break
            km.update_centers()
        tot[v] = s
        km.close()
    assert tot["elkan"] < tot["standard"] and tot["hamerly"] < tot["standard"]
    assert tot["yinyang"] < tot["standard"]


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_half_precision_values(dtype):
    """FP16 / BF16 stored values: the oracle promotes the same stored values."""
    base = synth.tfidf(synth.scaled(synth.CSR_TINY, n=1500, seed=7))
    if dtype == "f16":
        val = base.val.astype(np.float16)
        tval = torch.from_numpy(val).cuda()
        oval = val.astype(np.float64)
    else:
        tval = torch.from_numpy(base.val).to(torch.bfloat16).cuda()
        oval = tval.float().cpu().numpy().astype(np.float64)
    csr = synth.CSR(base.n, base.d, base.row_ptr, base.col, oval.astype(np.float32))
    init = synth.init_rows(csr.n, 16, 4)
    dev = (torch.from_numpy(base.row_ptr).cuda(), torch.from_numpy(base.col).cuda(), tval)
    X = oracle.Data(csr.n, csr.d, False, csr.row_ptr, csr.col, oval)
    ri = oracle.rinv(X)
    km = _km(csr, 16, "elkan", init, dev)
    prev = np.full(csr.n, -1, np.int32)
    for _ in range(6):
        C = km.centers()
        ch = km.assign()
        lab = km.labels()
        _check_assign(X, ri, C, prev, lab)
        if ch == 0:
            break
        km.update_centers()
        Co, _, _ = oracle.update(X, ri, lab, C.astype(np.float64))
        assert np.max(np.linalg.norm(km.centers() - Co, axis=1)) < CTOL
        prev = lab
    km.close()


def test_host_input_matches_device_input(tiny):
    init = synth.init_rows(tiny.n, 20, 1)
    a = _km(tiny, 20, "elkan", init)
    b = skm.KMeans(tiny.n, tiny.d, tiny.row_ptr, tiny.col, tiny.val, 20, variant="elkan", init_rows=init)
    ia, Ja = a.run(20)
    ib, Jb = b.run(20)
    assert ia == ib and Ja == Jb
    np.testing.assert_array_equal(a.labels(), b.labels())
    np.testing.assert_array_equal(a.centers(), b.centers())


def test_edge_cases():
    rng = np.random.default_rng(0)
    # rows of 1 nnz, rows longer than one 32-entry chunk, a term used by no row
    n, d = 300, 400
    dense = np.zeros((n, d), dtype=np.float32)
    for i in range(n):
        m = 1 if i % 7 == 0 else (70 if i % 11 == 0 else int(rng.integers(2, 20)))
        cols = rng.choice(d - 1, size=m, replace=False)
        dense[i, cols] = rng.uniform(0.1, 1.0, size=m)
    csr = synth.csr_from_dense(dense)
    X = oracle.Data.from_csr(csr)
    for k in (1, 2, 33, n):
        init = synth.init_rows(n, k, 9)
        for v in ["standard", "hamerly", "elkan"]:
            tr = oracle.run(X, oracle.unit_rows(X, init), v, max_iters=10)
            km = _km(csr, k, v, init)
            it, J = km.run(10)
            assert it == tr.iters
            lab = km.labels()
            np.testing.assert_array_equal(lab, tr.labels[-1])
            assert abs(J - tr.J[-1]) <= CTOL * abs(tr.J[-1])
            km.close()


def test_invalid_inputs_rejected():
    csr = synth.csr_from_dense(np.eye(6, dtype=np.float32))
    bad_col = csr.col.copy()
    bad_col[3] = 99
    with pytest.raises(skm.SkmError):
        skm.KMeans(6, 6, torch.from_numpy(csr.row_ptr).cuda(), torch.from_numpy(bad_col).cuda(),
                   torch.from_numpy(csr.val).cuda(), 2)
    zero = csr.val.copy()
    zero[2] = 0.0
    with pytest.raises(skm.SkmError):
        skm.KMeans(6, 6, torch.from_numpy(csr.row_ptr).cuda(), torch.from_numpy(csr.col).cuda(),
                   torch.from_numpy(zero).cuda(), 2)
    with pytest.raises(skm.SkmError):
        _km(csr, 2, "standard", [1, 1])


def test_incremental_sums_equal_full_recompute(mid):
    """Optimisation (iii) of Section 5: updating the sums with only the rows
    that moved gives bit for bit the centers of a full recomputation (the sums
    are exact fixed-point integers)."""
    init = synth.init_rows(mid.n, 100, 6)
    dev = _dev(mid)
    inc = _km(mid, 100, "elkan", init, dev)
    ref = _km(mid, 100, "standard", init, dev)
    for it in range(14):
        ch = inc.assign()
        lab = inc.labels()
        ref.set_labels(lab)            # forces a full recomputation of the sums
        ref.set_centers(inc.centers())
        if ch == 0:
            break
        Ji = inc.update_centers()
        Jr = ref.update_centers()
        np.testing.assert_array_equal(inc.centers(), ref.centers())
        assert Ji == Jr
    # an update with no assignment in between changes nothing
    C = inc.centers()
    inc.update_centers()
    np.testing.assert_array_equal(inc.centers(), C)
    inc.close()
    ref.close()


@pytest.mark.parametrize("variant", ["elkan", "simp_elkan"])
def test_long_rows_elkan(variant):
    """Rows of 200-2000 entries: the Elkan survivors go to the warp-per-point
    recompute (rows above 256 entries) as well as the 8-lane one.  Teacher-
    forced against the oracle, and bit for bit the standard variant's labels
    at every iteration."""
    cfg = synth.SparseCfg(n=3000, d=8000, seed=31, nnz_kind=1, a=600.0, b=0.5, lo=200, hi=2000, zipf=1.1)
    csr = synth.tfidf(cfg)
    assert np.mean(np.diff(csr.row_ptr) > 256) > 0.5
    init = synth.init_rows(csr.n, 40, 31)
    seq = _teacher_forced(csr, 40, variant, init, 25)
    std = _km(csr, 40, "standard", init)
    km = _km(csr, 40, variant, init)
    survivors = 0
    for t in range(len(seq)):
        ch = km.assign()
        std.assign()
        survivors += km.stats().last_survivors
        np.testing.assert_array_equal(km.labels(), std.labels())
        np.testing.assert_array_equal(km.labels(), seq[t])
        if ch == 0:
            break
        assert km.update_centers() == std.update_centers()
    assert survivors > 0  # the per-pair recompute ran
    km.close()
    std.close()


@pytest.mark.parametrize("variant", ["elkan", "simp_elkan"])
def test_elkan_bound_pass_schedule_keeps_labels(mid, variant):
    """While nearly every point goes to a whole row, Elkan's bound pass is
    skipped (every point goes straight to the whole-row pass, which rewrites
    its bounds) and run again every 8th iteration.  Labels and changed counts
    equal the standard variant's at every iteration; skipped iterations
    report last_skipped = 1 with every point recomputed whole, and later
    iterations pass the bounds again and prune."""
    k = 100
    init = synth.init_rows(mid.n, k, 2)
    dev = _dev(mid)
    std = _km(mid, k, "standard", init, dev)
    elk = _km(mid, k, variant, init, dev)
    skipped = pruned = 0
    for it in range(60):
        cs = std.assign()
        ch = elk.assign()
        assert ch == cs
        np.testing.assert_array_equal(elk.labels(), std.labels())
        st = elk.stats()
        if st.last_skipped:
            skipped += 1
            assert st.last_rechecks == mid.n and st.last_survivors == 0
        elif it > 0 and st.last_rechecks < mid.n // 2:
            pruned += 1
        if cs == 0:
            break
        std.update_centers()
        elk.update_centers()
    std.close()
    elk.close()
    assert skipped > 0 and pruned > 0


@pytest.mark.parametrize("variant", ["hamerly", "simp_hamerly"])
def test_hamerly_tightening_schedule_keeps_labels(mid, variant):
    """Where tightening prunes almost nothing, Hamerly's survivors go straight
    to the whole-row pass, with tightening again every 8th iteration.  The
    labels equal the standard variant's at every iteration, and the counters
    show both kinds of iteration: with at least 1024 survivors, a skipped one
    computes only whole rows (sims = rechecks k), a tightened one also one
    similarity per survivor (sims = survivors + rechecks k)."""
    k = 100
    init = synth.init_rows(mid.n, k, 2)
    dev = _dev(mid)
    std = _km(mid, k, "standard", init, dev)
    ham = _km(mid, k, variant, init, dev)
    skipped = tightened = 0
    for it in range(40):
        cs = std.assign()
        ch = ham.assign()
        assert ch == cs
        np.testing.assert_array_equal(ham.labels(), std.labels())
        st = ham.stats()
        if it > 0 and st.last_survivors >= 1024:
            if st.last_sims == st.last_rechecks * k:
                skipped += 1
            else:
                assert st.last_sims == st.last_survivors + st.last_rechecks * k
                tightened += 1
        if cs == 0:
            break
        std.update_centers()
        ham.update_centers()
    std.close()
    ham.close()
    assert skipped > 0 and tightened > 1


@pytest.mark.parametrize("variant,k,tiles", [("standard", 300, (128, 256)), ("elkan", 300, (128, 256)),
                                             ("simp_hamerly", 300, (256,)), ("simp_elkan", 1000, (512,))])
def test_center_tiles_give_the_same_run(variant, k, tiles):
    """The whole-row kernel walks a row once per tile of centers: with tiles
    smaller than the default, every iteration's labels, changed counts and
    objective are those of the default tile (FP16 screening on, as by default
    for k > 128)."""
    X = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=6000, d=8000, seed=41))
    init = synth.init_rows(X.n, k, 41)
    dev = _dev(X)
    runs = {}
    for kt in (0,) + tuple(tiles):
        km = _km(X, k, variant, init, dev, k_tile=kt)
        seq = []
        for _ in range(25):
            ch = km.assign()
            lab = km.labels()
            if ch == 0:
                seq.append((ch, lab, None))
                break
            seq.append((ch, lab, km.update_centers()))
        km.close()
        runs[kt] = seq
    for kt in tiles:
        assert len(runs[kt]) == len(runs[0])
        for (ca, la, ja), (cb, lb_, jb) in zip(runs[0], runs[kt]):
            assert ca == cb
            np.testing.assert_array_equal(la, lb_)
            assert ja == jb


def test_autotune_single_run_tiles_and_cache(tmp_path):
    """skm_autotune on a single run with k = 300 (default tile 512, screening
    on): it times the launch shapes, two smaller tiles and the screened pass
    off, writes one five-field cache line, a second context reads it back,
    and a run after either gives the labels of a default context."""
    X = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=6000, d=8000, seed=43))
    k = 300
    init = synth.init_rows(X.n, k, 43)
    dev = _dev(X)
    ref = _km(X, k, "simp_elkan", init, dev)
    it_ref, _ = ref.run(30)
    lab_ref = ref.labels()
    ref.close()
    cache = tmp_path / "tune.txt"
    a = _km(X, k, "simp_elkan", init, dev)
    assert a.autotune(cache, iters=2) is False
    f = cache.read_text().split()
    assert len(f) == 5 and int(f[3]) in (0, 128, 256) and int(f[4]) in (0, 1)
    it_a, _ = a.run(30)
    np.testing.assert_array_equal(a.labels(), lab_ref)
    assert it_a == it_ref
    a.close()
    b = _km(X, k, "simp_elkan", init, dev)
    assert b.autotune(cache, iters=2) is True
    it_b, _ = b.run(30)
    np.testing.assert_array_equal(b.labels(), lab_ref)
    b.close()


@pytest.mark.parametrize("variant", ["standard", "hamerly", "elkan", "simp_elkan"])
def test_fused_center_update_equals_separate_kernels(variant):
    """The center update's phases after the sums run as one cooperative
    launch (grid barriers between phases) or as separate kernels: labels,
    objective and centers are bit-identical at every iteration, eagerly and
    with the iteration replayed as a CUDA graph."""
    X = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=8000, d=6000, seed=23))
    k = 50
    init = synth.init_rows(X.n, k, 23)
    dev = [torch.from_numpy(a).cuda() for a in (X.row_ptr, X.col, X.val)]
    seqs = {}
    for sep in (False, True):
        km = skm.KMeans(X.n, X.d, *dev, k, variant=variant, init_rows=init, fused_update=not sep)
        seq = []
        for _ in range(40):
            ch = km.assign()
            lab = km.labels()
            if ch == 0:
                seq.append((lab, None, None))
                break
            J = km.update_centers()
            seq.append((lab, J, km.centers()))
        seqs[sep] = seq
        km.close()
    assert len(seqs[False]) == len(seqs[True])
    for (la, ja, ca), (lb, jb, cb) in zip(seqs[False], seqs[True]):
        np.testing.assert_array_equal(la, lb)
        assert ja == jb
        if ca is not None:
            np.testing.assert_array_equal(ca, cb)
    g = skm.KMeans(X.n, X.d, *dev, k, variant=variant, init_rows=init, graph=True, fused_update=True)
    it, J = g.run(40)
    assert it == len(seqs[True])
    np.testing.assert_array_equal(g.labels(), seqs[True][-1][0])
    g.close()


@pytest.mark.parametrize("k,screen", [(37, True), (300, None), (1000, None)])
@pytest.mark.parametrize("variant", ["elkan", "simp_elkan", "hamerly", "simp_hamerly"])
def test_screened_whole_rows_keep_the_standard_labels(k, screen, variant):
    """The Elkan and Hamerly variants screen their whole-row recomputes
    against FP16 centers (on by default for k > 128, forced on here for
    k = 37): a proven per-row bound decides most rows and the rest are
    recomputed exactly, so the label sequence over a whole run equals the
    standard variant's; the screened pass runs in every iteration after the
    first, and the bounds it leaves hold against exact similarities."""
    X = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=12000, d=9000, seed=29))
    init = synth.init_rows(X.n, k, 29)
    dev = _dev(X)
    seqs, prof = {}, {}
    for v in ("standard", variant):
        km = _km(X, k, v, init, dev, **({} if v == "standard" else {"screen": screen}))
        labs = []
        km.profile(True)
        for t in range(25):
            ch = km.assign()
            labs.append(km.labels())
            if ch == 0 or t == 24:  # stop right after an assignment: the bounds refer to these centers
                break
            km.update_centers()
        prof[v] = km.profile_read()
        km.profile(False)
        seqs[v] = labs
        if v == variant:
            C = km.centers().astype(np.float64)
            l, u = km.bounds()
            lab = km.labels()
            rows = np.random.default_rng(3).choice(X.n, 800, replace=False)
            sub = X.rows(rows)
            Xs = sub.dense() * oracle.rinv(oracle.Data.from_csr(sub))[:, None]
            S = Xs @ (C / np.linalg.norm(C, axis=1, keepdims=True)).T
            assert np.all(l[rows] <= S[np.arange(len(rows)), lab[rows]] + 1e-12)
            mask = np.ones_like(S, dtype=bool)
            mask[np.arange(len(rows)), lab[rows]] = False
            if u.ndim == 2:
                assert np.all(u[rows][mask] >= S[mask] - 1e-12)
            else:
                S2 = np.where(mask, S, -np.inf)
                assert np.all(u[rows] >= S2.max(axis=1) - 1e-12)
        km.close()
    assert len(seqs[variant]) == len(seqs["standard"])
    for a_, b_ in zip(seqs[variant], seqs["standard"]):
        np.testing.assert_array_equal(a_, b_)
    assert prof[variant]["k_rows_top2(screen)"][1] >= 1


def test_screened_teacher_forced():
    X = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=5000, d=6000, seed=31))
    init = synth.init_rows(X.n, 300, 31)
    _teacher_forced(X, 300, "elkan", init, 10, sample=1500)


def test_screening_off_gives_the_same_run():
    """screen off (exact FP32 whole rows) and on: identical labels and centers
    over a whole run at k = 300."""
    X = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=8000, d=7000, seed=33))
    init = synth.init_rows(X.n, 300, 33)
    dev = _dev(X)
    out = {}
    for scr in (False, True):
        km = _km(X, 300, "simp_elkan", init, dev, screen=scr)
        out[scr] = (km.run(40), km.labels(), km.centers())
        km.close()
    assert out[False][0] == out[True][0]
    np.testing.assert_array_equal(out[False][1], out[True][1])
    np.testing.assert_array_equal(out[False][2], out[True][2])
