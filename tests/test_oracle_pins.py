"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: brute force
with numpy on tiny inputs, closed forms, geometric constructions, invariants
the paper states, and the numbers the paper prints.  Together they are chosen
so that a dropped term, a wrong sign, a wrong index or a transposed operand in
the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
VARIANTS = ["standard", "hamerly", "elkan", "simp_hamerly", "simp_elkan", "yinyang"]


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _brute_labels(Xn, C, cur):
    """Dense brute force: all n*k cosines, argmax under the tie rule."""
    S = Xn @ C.T
    out = np.empty(len(Xn), dtype=np.int32)
    for i in range(len(Xn)):
        m = S[i].max()
        if cur[i] >= 0 and S[i, cur[i]] == m:
            out[i] = cur[i]
        else:
            out[i] = int(np.flatnonzero(S[i] == m)[0])
    return out


# ------------------------------------------------------------- assignment

@pytest.mark.parametrize("seed", range(6))
def test_assign_matches_brute_force(seed):
    """Section 5: a(i) = argmax_j <x(i), c(j)> -- oracle vs dense numpy."""
    rng = np.random.default_rng(seed)
    n, d, k = int(rng.integers(5, 64)), int(rng.integers(2, 16)), int(rng.integers(1, 6))
    Xs = rng.standard_normal((n, d)) * rng.uniform(0.5, 3.0, size=(n, 1))
    Xs[rng.random((n, d)) < 0.3] = 0.0
    Xs[:, 0] += 1e-3  # no zero rows
    C = _unit(rng.standard_normal((k, d)))
    for dense in (True, False):
        X = oracle.Data.from_dense(Xs) if dense else oracle.Data.from_csr(synth.csr_from_dense(Xs))
        ri = oracle.rinv(X)
        Xn = Xs / np.linalg.norm(Xs, axis=1, keepdims=True) if dense else \
            synth.csr_from_dense(Xs).dense() * ri[:, None]
        cur = rng.integers(-1, k, size=n).astype(np.int32)
        lab, ch, sb, ss, gap = oracle.assign(X, ri, C, cur)
        want = _brute_labels(Xn, C, cur)
        np.testing.assert_array_equal(lab, want)
        assert ch == int(np.sum(want != cur))
        S = Xn @ C.T
        np.testing.assert_allclose(sb, S[np.arange(n), want], rtol=0, atol=1e-13)
        srt = np.sort(S, axis=1)
        if k > 1:
            np.testing.assert_allclose(gap, srt[:, -1] - srt[:, -2], atol=1e-13)


def test_tie_rule_on_exact_integer_dots():
    """Reading T on exact ties: integer vectors whose dots are exact in FP64."""
    # rows e0, e1, e0+e1 (normalised); centers e0, e1 -> row 2 ties.
    Xs = np.array([[1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 0, 1]], dtype=np.float64)
    C = np.eye(3)[:2]
    X = oracle.Data.from_dense(Xs)
    ri = oracle.rinv(X)
    lab, ch, *_ = oracle.assign(X, ri, C)              # no current label
    assert lab.tolist() == [0, 1, 0, 0]                 # lowest index wins; row 3 ties at 0
    lab, ch, *_ = oracle.assign(X, ri, C, np.array([1, 0, 1, 1], dtype=np.int32))
    assert lab.tolist() == [0, 1, 1, 1]                 # current label wins a tie
    assert ch == 2


# ----------------------------------------------------------- center update

@pytest.mark.parametrize("seed", range(4))
def test_update_closed_form(seed):
    """Section 5: c(j) = sum / |sum|; empty clusters keep their center."""
    rng = np.random.default_rng(100 + seed)
    n, d, k = 40, 7, 5
    Xs = np.abs(rng.standard_normal((n, d))) * rng.uniform(0.2, 2, size=(n, 1))
    X = oracle.Data.from_dense(Xs)
    ri = oracle.rinv(X)
    Xn = Xs / np.linalg.norm(Xs, axis=1, keepdims=True)
    a = rng.integers(0, k - 1, size=n).astype(np.int32)  # cluster k-1 empty
    C_old = _unit(rng.standard_normal((k, d)))
    Cn, norms, J = oracle.update(X, ri, a, C_old)
    S = np.zeros((k, d))
    np.add.at(S, a, Xn)
    for j in range(k - 1):
        np.testing.assert_allclose(Cn[j], S[j] / np.linalg.norm(S[j]), atol=1e-15)
    np.testing.assert_array_equal(Cn[k - 1], C_old[k - 1])
    np.testing.assert_allclose(np.linalg.norm(Cn, axis=1), 1.0, atol=1e-15)
    # J = sum_j |S_j| = sum_i <x_i, c_a(i)>
    assert J == pytest.approx(np.linalg.norm(S, axis=1).sum(), rel=1e-14)
    assert J == pytest.approx(float(np.sum(Xn * Cn[a])), rel=1e-13)


def test_worked_circle_example():
    """A hand-derived case: six unit vectors on a circle in two groups."""
    g = json.load(open(os.path.join(GOLDEN, "circle_worked.json")))
    ang = np.deg2rad(g["angles_deg"])
    Xs = np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], axis=1) * 2.5  # unnormalised on purpose
    X = oracle.Data.from_dense(Xs)
    ri = oracle.rinv(X)
    C0 = Xs[g["init_rows"]] / 2.5
    tr = oracle.run(X, C0, "standard", max_iters=10)
    assert tr.labels[0].tolist() == g["labels"]
    want = np.deg2rad(g["center_angles_deg"])
    np.testing.assert_allclose(tr.C[:, 0], np.cos(want), atol=1e-14)
    np.testing.assert_allclose(tr.C[:, 1], np.sin(want), atol=1e-14)
    assert tr.J[0] == pytest.approx(eval(g["J_closed_form"], {"cos": math.cos, "radians": math.radians}), rel=1e-14)
    assert tr.iters == 2 and tr.changed.tolist() == [6, 0]


# --------------------------------------------------------------- identities

def test_cosine_euclid_identity(tiny_csr):
    """Eq. (eqn:euclid): sim = 1 - d^2/2 on unit vectors (Section 2)."""
    X = oracle.Data.from_csr(tiny_csr)
    ri = oracle.rinv(X)
    Xd = tiny_csr.dense() * ri[:, None]
    rng = np.random.default_rng(7)
    for _ in range(50):
        i, j = rng.integers(0, tiny_csr.n, size=2)
        s = oracle.sim(X, ri, i, Xd[j])
        dist2 = float(np.sum((Xd[i] - Xd[j]) ** 2))
        assert s == pytest.approx(1.0 - 0.5 * dist2, abs=1e-14)


@pytest.mark.parametrize("phi", [1e-7, 1e-4, 0.3, 1.2, 2.5, math.pi])
def test_drift_closed_form(phi):
    """p = cos(phi) and its sine for two unit vectors at angle phi (Section 4),
    including tiny angles where 1 - p^2 cancels."""
    rng = np.random.default_rng(3)
    e1 = _unit(rng.standard_normal(9))
    e2 = rng.standard_normal(9)
    e2 = _unit(e2 - e2 @ e1 * e1)
    a = e1
    b = math.cos(phi) * e1 + math.sin(phi) * e2
    p, sp = oracle.drift(a[None], b[None])
    assert p[0] == pytest.approx(math.cos(phi), abs=1e-15)
    assert sp[0] == pytest.approx(math.sin(phi), rel=1e-9, abs=1e-15)


@pytest.mark.parametrize("phi", [0.0, 0.4, 1.0, 2.0, 3.0])
def test_half_angle_center_bound(phi):
    """Section 5.2: cc = sqrt((<c_i,c_j>+1)/2) = cos(phi/2); s = max over others."""
    C = np.array([[1.0, 0.0, 0.0], [math.cos(phi), math.sin(phi), 0.0], [0.0, 0.0, 1.0]])
    cc, s = oracle.center_bounds(C)
    assert cc[0, 1] == pytest.approx(math.cos(phi / 2), abs=1e-14)
    assert cc[1, 0] == pytest.approx(math.cos(phi / 2), abs=1e-14)
    assert cc[0, 2] == pytest.approx(math.cos(math.pi / 4), abs=1e-14)
    assert s[2] == pytest.approx(math.cos(math.pi / 4), abs=1e-14)
    assert s[0] == pytest.approx(max(math.cos(phi / 2), math.cos(math.pi / 4)), abs=1e-14)


def test_elkan_center_test_is_valid():
    """Section 5.2: if cc(a,j) <= l <= <x,c_a> and l >= 0 then <x,c_j> <= l.
    Checked on random geometric configurations (with the oracle's cc)."""
    rng = np.random.default_rng(11)
    hits = 0
    for _ in range(4000):
        d = 5
        x, ca, cj = _unit(rng.standard_normal((3, d)))
        ca = _unit(x + rng.uniform(0, 1.5) * ca)
        l = float(x @ ca)
        cc, _ = oracle.center_bounds(np.stack([ca, cj]))
        if l >= 0 and cc[0, 1] <= l:
            hits += 1
            assert float(x @ cj) <= l + 1e-12
    assert hits > 100


def test_elkan_derivation_reaches_l():
    """Section 5.2: with <c_a,c_j> = 2l^2-1 the cosine bound equals l exactly:
    realised by x at angle t from c_a and c_j at angle 2t on the far side."""
    for t in np.linspace(0.01, math.pi / 2, 25):
        x = np.array([1.0, 0.0])
        ca = np.array([math.cos(t), math.sin(t)])
        cj = np.array([math.cos(-t), math.sin(-t)])     # angle 2t from c_a
        l = float(x @ ca)
        cc, _ = oracle.center_bounds(np.stack([ca, cj]))
        assert float(ca @ cj) == pytest.approx(2 * l * l - 1, abs=1e-14)
        assert cc[0, 1] == pytest.approx(l, abs=1e-12)   # half-angle = t
        assert float(x @ cj) == pytest.approx(l, abs=1e-14)  # the bound is attained


# ----------------------------------------------------------- bound algebra

def test_bounds_match_arc_length_form():
    """Eq. (eqn:l-bound)/(eqn:u-elkan) equal the arc-length triangle
    inequality Eq. (eq:tri-acos) evaluated with libm (Section 3)."""
    rng = np.random.default_rng(5)
    for _ in range(3000):
        l, u, p = rng.uniform(-1, 1, size=3)
        tl, tu, tp = math.acos(l), math.acos(u), math.acos(p)
        want_l = math.cos(tl + tp) if tl + tp <= math.pi else -1.0
        want_u = math.cos(max(0.0, tu - tp))
        assert oracle.l_update(l, p) == pytest.approx(want_l, abs=1e-12)
        assert oracle.l_update(l, p) <= want_l + 1e-15
        assert oracle.u_update(u, p) == pytest.approx(want_u, abs=1e-12)
        assert oracle.u_update(u, p) >= want_u - 1e-15


def test_bounds_valid_on_geometry():
    """The updated bounds hold for actual vectors: x, c, c' on a sphere."""
    rng = np.random.default_rng(6)
    for _ in range(3000):
        x, c, c2 = _unit(rng.standard_normal((3, 4)))
        c2 = _unit(c + rng.uniform(0, 2) * c2)
        s_old, s_new, p = float(x @ c), float(x @ c2), float(c @ c2)
        lo = s_old - rng.uniform(0, 0.3)   # any valid lower bound
        hi = s_old + rng.uniform(0, 0.3)   # any valid upper bound
        lo, hi = max(lo, -1.0), min(hi, 1.0)
        assert oracle.l_update(lo, p) <= s_new + 1e-12
        assert oracle.u_update(hi, p) >= s_new - 1e-12


def test_clamp_counterexample():
    """Reading CL: u = 0.5, p = 0.3.  The unclamped Eq. (eqn:u-elkan) gives
    0.976, yet x with <x,c> = 0.3 <= u and c' = x (so <c,c'> = 0.3) reaches 1."""
    u, p = 0.5, 0.3
    raw = u * p + math.sqrt((1 - u * u) * (1 - p * p))
    assert raw == pytest.approx(0.976, abs=1e-3)
    x = np.array([1.0, 0.0])
    c = np.array([0.3, math.sqrt(1 - 0.09)])
    c2 = x.copy()
    assert float(x @ c) <= u and float(c @ c2) == pytest.approx(p)
    assert oracle.u_update(u, p) >= float(x @ c2) == 1.0


def test_hamerly_pitfall_and_guard():
    """Section 5.3: the single-center update is not minimised by the
    smallest p (u = 0.99, p in {0.5, 0.99}); Eq. (eqn:u-hamerly-2) covers
    both; reading HG: with p' = -0.99 it would give 0.961 < 1 = the valid
    bound, so the guard must fall back to the clamped form."""
    raw = lambda u, p: u * p + math.sqrt((1 - u * u) * (1 - p * p))
    assert raw(0.99, 0.5) == pytest.approx(0.617, abs=1e-3)
    assert raw(0.99, 0.99) == pytest.approx(1.0, abs=1e-12)
    assert raw(0.99, 0.5) < raw(0.99, 0.99)            # the pitfall
    h = oracle.u_hamerly(0.99, 0.5)
    assert h >= 1.0 - 1e-15
    paper = 0.9 + math.sqrt((1 - 0.81) * (1 - 0.99 ** 2))
    assert paper == pytest.approx(0.961, abs=1e-3)
    assert oracle.u_hamerly(0.9, -0.99) == 1.0


def test_hamerly_bound_dominates_every_center():
    """u_hamerly(u, min p) >= the per-center bound for every p >= min p."""
    rng = np.random.default_rng(8)
    for _ in range(3000):
        u = float(rng.uniform(-1, 1))
        ps = rng.uniform(-1, 1, size=6)
        for tight in (False, True):
            h = oracle.u_hamerly(u, float(ps.min()), tight=tight)
            for p in ps:
                assert h >= oracle.u_update(u, float(p)) - 1e-15


def test_u_update_grows_as_drift_grows():
    """Yin-Yang's group bound moves with the group's smallest p: Eq.
    (eqn:u-elkan) with the clamp never decreases when p decreases, so that
    update bounds every center of the group."""
    rng = np.random.default_rng(12)
    for _ in range(4000):
        u = rng.uniform(-1, 1)
        p1, p2 = np.sort(rng.uniform(-1, 1, 2))
        assert oracle.u_update(u, p1) >= oracle.u_update(u, p2) - 1e-15
    # and against the arc form: cos(max(0, arccos u - arccos p)) is the bound for one center
    for u in np.linspace(-0.99, 0.99, 41):
        for pp in np.linspace(-0.99, 0.99, 41):
            want = np.cos(max(0.0, np.arccos(u) - np.arccos(pp)))
            assert abs(oracle.u_update(u, pp) - want) < 1e-9


# ------------------------------------------------------------- full runs

def _runs(X, C0, max_iters, **kw):
    return {v: oracle.run(X, C0, v, max_iters=max_iters, **kw) for v in VARIANTS}


def test_variants_identical_labels_sparse(tiny_csr):
    """Section 4: pruning only skips provably unnecessary similarities, so all
    variants produce the standard variant's label sequence."""
    X = oracle.Data.from_csr(tiny_csr)
    C0 = oracle.unit_rows(X, synth.init_rows(tiny_csr.n, 20, 1))
    runs = _runs(X, C0, 20, check_bounds=True)
    ref = runs["standard"]
    for v, tr in runs.items():
        assert tr.violations == 0, v
        assert tr.iters == ref.iters
        np.testing.assert_array_equal(tr.labels, ref.labels)
        np.testing.assert_allclose(tr.J, ref.J, rtol=1e-13)
        if v != "standard":
            assert tr.sims.sum() < ref.sims.sum()


@pytest.mark.parametrize("tight", [False, True])
def test_variants_identical_labels_dense(tight):
    """Same on dense vMF data, where many iterations and sign changes occur."""
    Xs, comp, _ = synth.vmf(1500, 24, 12, 8.0, seed=21, return_comp=True)
    X = oracle.Data.from_dense(Xs)
    C0 = oracle.unit_rows(X, synth.init_rows(1500, 12, 21))
    runs = _runs(X, C0, 60, check_bounds=True, hamerly_tight=tight)
    ref = runs["standard"]
    assert ref.iters > 5
    for v, tr in runs.items():
        assert tr.violations == 0, v
        np.testing.assert_array_equal(tr.labels, ref.labels)
    # Elkan needs the fewest similarity computations (Section 6, Fig. 1)
    assert runs["elkan"].sims.sum() <= runs["hamerly"].sims.sum()


def test_objective_non_decreasing():
    """Alternating maximisation (Section 5): J never decreases."""
    Xs = synth.vmf(2000, 16, 30, 5.0, seed=4)
    X = oracle.Data.from_dense(Xs)
    C0 = oracle.unit_rows(X, synth.init_rows(2000, 30, 4))
    tr = oracle.run(X, C0, "standard", max_iters=50)
    assert tr.iters > 3
    assert np.all(np.diff(tr.J) >= -1e-12 * tr.J[1:])


# ---------------------------------------------------------- special cases

def test_k_equals_one():
    """k = 1: every label 0, the center is the normalised global sum."""
    Xs = np.abs(np.random.default_rng(1).standard_normal((30, 6)))
    X = oracle.Data.from_dense(Xs)
    C0 = oracle.unit_rows(X, [3])
    for v in VARIANTS:
        tr = oracle.run(X, C0, v, max_iters=5)
        assert np.all(tr.labels == 0)
        tot = (Xs / np.linalg.norm(Xs, axis=1, keepdims=True)).sum(0)
        np.testing.assert_allclose(tr.C[0], tot / np.linalg.norm(tot), atol=1e-15)


def test_k_equals_n_distinct_rows():
    """k = n with distinct rows: every row is its own center; one update later
    nothing changes."""
    Xs = np.abs(np.random.default_rng(2).standard_normal((12, 5))) + 0.1
    X = oracle.Data.from_dense(Xs)
    C0 = oracle.unit_rows(X, np.arange(12))
    for v in VARIANTS:
        tr = oracle.run(X, C0, v, max_iters=5)
        assert tr.labels[0].tolist() == list(range(12))
        assert tr.changed.tolist() == [12, 0]


def test_antipodal_clusters():
    """Two well separated antipodal groups get their known labels."""
    rng = np.random.default_rng(9)
    A = _unit(np.array([1.0, 0, 0, 0]) + 0.05 * rng.standard_normal((20, 4)))
    B = _unit(np.array([-1.0, 0, 0, 0]) + 0.05 * rng.standard_normal((20, 4)))
    Xs = np.concatenate([A, B])
    X = oracle.Data.from_dense(Xs)
    C0 = oracle.unit_rows(X, [0, 1])        # both seeds in group A
    for v in VARIANTS:
        tr = oracle.run(X, C0, v, max_iters=20)
        lab = tr.labels[-1]
        assert len(set(lab[:20])) == 1 and len(set(lab[20:])) == 1 and lab[0] != lab[20]


def test_orthonormal_rows_tie_rule():
    """Rows e_i: all cross similarities are 0, so the tie rule decides."""
    Xs = np.eye(8)
    X = oracle.Data.from_dense(Xs)
    C0 = oracle.unit_rows(X, [5, 2])
    lab, *_ = oracle.assign(X, oracle.rinv(X), C0)
    assert lab.tolist() == [0, 0, 1, 0, 0, 0, 0, 0]


# ------------------------------------------------------ paper's own numbers

def test_memory_figures_from_the_paper():
    """Section 6: for DBLP author-conference (Table 1) at k = 100, Hamerly adds
    44 MB (three 8-byte values per point) while Elkan's FP64 bounds need
    'about 2 GB' (n*k*8 bytes, 1.47 GB)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_figures.json")))
    n = g["dblp_author_conference"]["rows"]
    assert round(n * 3 * 8 / 1e6) == g["hamerly_bound_mb"]
    elkan = n * g["k"] * 8 / 1e9
    assert 1.0 < elkan < g["elkan_bound_gb_stated"]
    assert abs(elkan - 1.47) < 0.01


# ---------------------------------------------------------------- k-means++ seeding (Section 5.6)

def _unit_dense(X):
    X = np.asarray(X, dtype=np.float64)
    return X / np.linalg.norm(X, axis=1, keepdims=True)


def test_kmeanspp_first_center_is_uniform_draw():
    X = np.abs(np.random.default_rng(3).normal(size=(10, 4))) + 0.1
    d = oracle.Data.from_dense(X.astype(np.float32))
    ri = oracle.rinv(d)
    for u0, want in ((0.0, 0), (0.05, 0), (0.1, 1), (0.55, 5), (0.999, 9)):
        assert oracle.kmeanspp(d, ri, [u0])[0] == want


def test_kmeanspp_second_center_proportional_to_one_minus_cos():
    """Sweeping the second draw over a fine grid, each row is chosen for a
    share of the grid equal to (1 - cos(x_i, c_1)) / sum, the paper's weight,
    computed here directly from the normalised rows."""
    X = np.abs(np.random.default_rng(5).normal(size=(7, 5))) + 0.05
    d = oracle.Data.from_dense(X.astype(np.float32))
    ri = oracle.rinv(d)
    Xn = _unit_dense(X.astype(np.float32))
    u0 = 0.3  # first center: row 2
    w = 1.0 - Xn @ Xn[2]
    w = np.clip(w, 0.0, None)
    M = 20000
    counts = np.zeros(len(X))
    for m in range(M):
        r = oracle.kmeanspp(d, ri, [u0, (m + 0.5) / M])
        assert r[0] == 2
        counts[r[1]] += 1
    np.testing.assert_allclose(counts / M, w / w.sum(), atol=2.0 / M)
    assert counts[2] == 0  # the chosen row has weight 0


def test_kmeanspp_k_equals_n_chooses_every_row_once():
    X = np.abs(np.random.default_rng(8).normal(size=(12, 6))) + 0.01
    X[5] = X[3]  # an exact duplicate: weight 0 once its twin is chosen
    d = oracle.Data.from_dense(X.astype(np.float32))
    ri = oracle.rinv(d)
    rows = oracle.kmeanspp(d, ri, np.random.default_rng(1).random(12))
    assert sorted(rows.tolist()) == list(range(12))


def test_kmeanspp_spreads_over_separated_clusters():
    """Three tight, mutually orthogonal clusters: after one center, the other
    clusters carry all the weight, so three draws land in three clusters."""
    rng = np.random.default_rng(2)
    base = np.eye(3)
    X = np.concatenate([base[c] + 1e-3 * np.abs(rng.normal(size=(20, 3))) for c in range(3)])
    d = oracle.Data.from_dense(X.astype(np.float32))
    ri = oracle.rinv(d)
    for s in range(25):
        rows = oracle.kmeanspp(d, ri, np.random.default_rng(100 + s).random(3))
        assert len({int(r) // 20 for r in rows}) == 3
