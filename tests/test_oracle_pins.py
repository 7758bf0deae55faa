"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, library special functions in a special case, brute-force sums, Ewald
summation (exact periodic Coulomb energy), direct O(N^2) sums, invariants of
the algorithms.  A dropped term, a wrong sign, index or factor in the oracle
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import special

import oracle as O
from paper_2006_16622_gb300.workloads import rocksalt, uniform_system

pytestmark = pytest.mark.usefixtures("oracle_lib")

_GOLD = {}
with open(os.path.join(os.path.dirname(__file__), "golden", "constants.txt")) as f:
    for line in f:
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            _GOLD[k] = float(v)


def _random_dir(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------- harmonics
def test_ylm_special_case_is_associated_legendre():
    """Y_n^m = sqrt((n-|m|)!/(n+|m|)!) P_n^|m|(cos t) e^{i m phi}; scipy's lpmv
    carries the Condon-Shortley phase (-1)^m, which the convention drops."""
    p = 12
    rng = np.random.default_rng(0)
    for _ in range(5):
        th, ph = rng.uniform(0, math.pi), rng.uniform(-math.pi, math.pi)
        Y = O.ylm(p, th, ph)
        for n in range(p + 1):
            for m in range(-n, n + 1):
                am = abs(m)
                ref = (math.sqrt(math.factorial(n - am) / math.factorial(n + am))
                       * (-1) ** am * special.lpmv(am, n, math.cos(th)) * np.exp(1j * m * ph))
                assert abs(Y[O.idx(n, m)] - ref) < 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("ratio", [0.2, 0.5, 0.8])
def test_addition_theorem_truncation_bound(ratio):
    """Eq. (2) with L_n^m = q r^-(n+1) Y_n^-m (Alg. L.2) is the Legendre
    expansion of 1/|x - y|; the truncation error obeys
    |err| <= (r/R)^(p+1) / (R - r)."""
    rng = np.random.default_rng(1)
    for p in (4, 10, 20, 30):
        for _ in range(3):
            y = 2.0 * _random_dir(rng)
            x = ratio * 2.0 * _random_dir(rng)
            irr = O.irregular(p, y)
            Lc = np.array([irr[O.idx(n, -m)] for n in range(p + 1) for m in range(-n, n + 1)])
            approx = O.eval_local(p, Lc, x)
            exact = 1.0 / np.linalg.norm(x - y)
            bound = ratio ** (p + 1) / (2.0 - 2.0 * ratio)
            assert abs(approx - exact) <= 1.01 * bound + 1e-14


def test_multipole_to_local_converges_to_direct():
    """M2L of Eq. (4) multipoles reproduces the direct potential of the
    cluster with error below the geometric bound."""
    rng = np.random.default_rng(2)
    src = rng.uniform(-0.5, 0.5, size=(12, 3))
    q = rng.choice([-1.0, 1.0], 12)
    c = np.array([3.0, 1.5, -2.0])
    x = rng.uniform(-0.5, 0.5, size=3)
    exact = sum(q[i] / np.linalg.norm(x - src[i] - c) for i in range(12))
    rs = np.max(np.linalg.norm(src, axis=1))
    ratio = (rs + np.linalg.norm(x)) / np.linalg.norm(c)
    prev = None
    for p in (4, 8, 12, 16, 20):
        M = O.multipole(p, src + c, q, c)
        err = abs(O.eval_local(p, O.m2l(p, M, c), x) - exact)
        bound = np.abs(q).sum() * ratio ** (p + 1) / (np.linalg.norm(c) * (1 - ratio))
        assert err <= bound + 1e-13
        if prev is not None and prev > 1e-13:
            assert err < prev
        prev = err
    assert prev < 1e-10


# -------------------------------------------------------------- lattice sums
def _lattice_sum_bruteforce(l, m, shells):
    g = np.arange(-shells, shells + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    keep = np.maximum(np.maximum(abs(X), abs(Y)), abs(Z)) >= 2
    X, Y, Z = X[keep].astype(float), Y[keep].astype(float), Z[keep].astype(float)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    th, ph = np.arccos(Z / r), np.arctan2(Y, X)
    am = abs(m)
    Ylm = (math.sqrt(math.factorial(l - am) / math.factorial(l + am)) * (-1) ** am
           * special.lpmv(am, l, np.cos(th)) * np.exp(1j * m * ph))
    return np.sum(Ylm / r ** (l + 1))


def test_lattice_sums_symmetry_zeros_and_cubic_ratios():
    lmax = 24
    S = O.lattice_sums(lmax)
    scale = max(abs(S))
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            v = S[O.idx(l, m)]
            if l <= 2 or l % 2 == 1 or m % 4 != 0:
                assert abs(v) <= 1e-13 * scale, (l, m, v)
            assert abs(v - np.conj(S[O.idx(l, -m)])) <= 1e-13 * scale
    r4 = S[O.idx(4, 4)].real / S[O.idx(4, 0)].real
    r6 = S[O.idx(6, 4)].real / S[O.idx(6, 0)].real
    assert abs(r4 - _GOLD["cubic_ratio_4"]) < 1e-11
    assert abs(r6 - _GOLD["cubic_ratio_6"]) < 1e-11


@pytest.mark.parametrize("l,m,tol", [(6, 0, 2e-6), (8, 0, 1e-8), (8, 4, 1e-8), (10, 8, 1e-9)])
def test_lattice_sums_match_direct_shell_summation(l, m, tol):
    """the Ewald-split value equals the plain cube-shell sum (tail bounded
    by the shells left out)"""
    S = O.lattice_sums(24)
    brute = _lattice_sum_bruteforce(l, m, 40)
    ref = S[O.idx(l, m)]
    assert abs(ref - brute) <= tol * abs(ref)


def test_lattice_sum_l4_extrapolated():
    """l = 4 converges like 1/shells^2: Richardson over two shell counts"""
    S = O.lattice_sums(8)[O.idx(4, 0)].real
    b1 = _lattice_sum_bruteforce(4, 0, 30).real
    b2 = _lattice_sum_bruteforce(4, 0, 60).real
    extrap = (4 * b2 - b1) / 3
    assert abs(extrap - S) < 2e-5 * abs(S)
    assert abs(extrap - S) < abs(b2 - S)


# -------------------------------------------------------------------- Ewald
@pytest.mark.parametrize("m", [4, 6])
def test_ewald_madelung_rocksalt(m):
    pos, q, a = rocksalt(m)
    U = O.ewald_energy(pos, q, a)
    assert abs(U / len(q) + _GOLD["madelung_nacl"] / 2) < 1e-12


# ------------------------------------------------------------ interaction list
def test_interaction_list_size_symmetry_and_tiling():
    pos, q = uniform_system(64, 8.0, seed=3)
    L = 4
    s = O.System(pos, q, 8.0, L, 2)
    assert int(_GOLD["il_size"]) == 189
    # sizes and symmetry on every level
    for lev in range(2, L + 1):
        n = 1 << (lev - 1)
        for cell in [(0, 0, 0), (n - 1, 0, n // 2), (n // 2, n - 1, n - 1)]:
            il = s.interaction_list(lev, cell)
            assert len(il) == 189
            cl = (cell[0] * n + cell[1]) * n + cell[2]
            for lin_b, sx, sy, sz in il:
                b = (lin_b // (n * n), (lin_b // n) % n, lin_b % n)
                back = s.interaction_list(lev, b)
                assert any(row[0] == cl and (row[1], row[2], row[3]) == (-sx, -sy, -sz)
                           for row in back)
    # the interaction lists of a finest cell's ancestors plus its 27 near
    # cells tile the 3^3 box copies exactly once
    nL = 1 << (L - 1)
    rng = np.random.default_rng(0)
    for _ in range(4):
        c = rng.integers(0, nL, 3)
        cover = {}
        for lev in range(2, L + 1):
            n = 1 << (lev - 1)
            f = 1 << (L - lev)
            anc = c >> (L - lev)
            for lin_b, sx, sy, sz in s.interaction_list(lev, anc):
                b = np.array((lin_b // (n * n), (lin_b // n) % n, lin_b % n))
                e = b + np.array((sx, sy, sz)) * n
                for dx in range(f):
                    for dy in range(f):
                        for dz in range(f):
                            k = (e[0] * f + dx, e[1] * f + dy, e[2] * f + dz)
                            cover[k] = cover.get(k, 0) + 1
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    k = (c[0] + dx, c[1] + dy, c[2] + dz)
                    cover[k] = cover.get(k, 0) + 1
        assert len(cover) == (3 * nL) ** 3
        assert all(v == 1 for v in cover.values())
        assert all(-nL <= k[i] < 2 * nL for k in cover for i in range(3))


def test_free_space_interaction_lists_skip_outside_cells():
    pos, q = uniform_system(64, 8.0, seed=3)
    s = O.System(pos, q, 8.0, 4, 2, bc=O.BC_FREE)
    assert len(s.interaction_list(2, (0, 1, 1))) == 0
    il = s.interaction_list(4, (0, 0, 0))
    assert 0 < len(il) < 189 and np.all(il[:, 1:] == 0)


def test_image_constant():
    acc = sum(1.0 / math.sqrt(x * x + y * y + z * z)
              for x in (-1, 0, 1) for y in (-1, 0, 1) for z in (-1, 0, 1) if (x, y, z) != (0, 0, 0))
    assert abs(acc - _GOLD["image_constant"]) < 1e-13
    assert int(_GOLD["n_images"]) == 26


# ------------------------------------------------------- energies and moves
def test_method_madelung_rocksalt():
    pos, q, a = rocksalt(8)
    s = O.System(pos, q, a, 3, 20)
    s.setup()
    assert abs(s.energy() / len(q) + _GOLD["madelung_nacl"] / 2) < 1e-8


def test_energy_converges_to_ewald_and_dipole_term():
    pos, q = uniform_system(32, 4.0, seed=5)
    a = 4.0
    Ue = O.ewald_energy(pos, q, a)
    errs = []
    for p in (8, 14, 20):
        s = O.System(pos, q, a, 3, p)
        s.setup()
        errs.append(abs(s.energy() - Ue))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6 * abs(Ue)
    sv = O.System(pos, q, a, 3, 14, dipole_bc=O.VACUUM)
    sv.setup()
    st = O.System(pos, q, a, 3, 14)
    st.setup()
    D = (q[:, None] * pos).sum(0)
    assert abs((sv.energy() - st.energy()) - 2 * math.pi / (3 * a ** 3) * D @ D) < 1e-12 * abs(Ue)


def test_propose_matches_ewald_difference():
    pos, q = uniform_system(32, 4.0, seed=6)
    a = 4.0
    rng = np.random.default_rng(7)
    s = O.System(pos, q, a, 3, 20)
    s.setup()
    for t in range(6):
        j = int(rng.integers(len(q)))
        rn = (pos[j] + rng.uniform(-0.8, 0.8, 3)) % a  # includes wraps
        dE = s.propose(j, rn)
        pos2 = pos.copy()
        pos2[j] = rn
        dEx = O.ewald_energy(pos2, q, a) - O.ewald_energy(pos, q, a)
        assert abs(dE - dEx) < 1e-6 * max(1.0, abs(dEx))
        # factored far field equals the literal form of Sec. 3.4 (iv)
        lit = s.last_parts()[2]
        assert abs(s.far_delta_factored(j, rn) - lit) < 1e-13 * max(1.0, abs(lit))
        if t % 2 == 0:
            s.accept(j, rn, dE)
            pos = pos2


def test_free_space_matches_direct_sums():
    pos, q = uniform_system(48, 8.0, seed=8)
    s = O.System(pos, q, 8.0, 4, 20, bc=O.BC_FREE)
    s.setup()
    Ud = O.direct_energy(pos, q)
    assert abs(s.energy() - Ud) < 1e-7 * abs(Ud)
    rng = np.random.default_rng(9)
    for _ in range(5):
        j = int(rng.integers(len(q)))
        rn = np.clip(pos[j] + rng.uniform(-1.5, 1.5, 3), 0.0, 7.999)
        dE = s.propose(j, rn)
        pos2 = pos.copy()
        pos2[j] = rn
        dEx = O.direct_energy(pos2, q) - Ud
        assert abs(dE - dEx) < 1e-7 * max(1.0, abs(dEx))
        s.accept(j, rn, dE)
        pos, Ud = pos2, Ud + dEx
    assert s.propose(0, np.array([8.5, 1.0, 1.0])) == math.inf


def test_free_space_move_back_antisymmetry():
    pos, q = uniform_system(200, 10.0, seed=10)
    s = O.System(pos, q, 10.0, 4, 10, bc=O.BC_FREE)
    s.setup()
    rng = np.random.default_rng(11)
    for _ in range(10):
        j = int(rng.integers(len(q)))
        r0 = s.positions()[j].copy()
        rn = np.clip(r0 + rng.uniform(-0.5, 0.5, 3), 0.0, 9.999)
        d1 = s.propose(j, rn)
        s.accept(j, rn, d1)
        d2 = s.propose(j, r0)
        assert abs(d1 + d2) <= 1e-12 * max(1.0, abs(d1))


def test_periodic_move_back_antisymmetry_falls_with_p():
    """with periodic images the moved charge's own images enter through the
    truncated level-2 expansions, so move-back antisymmetry holds to
    truncation and improves with p"""
    pos, q = uniform_system(64, 6.0, seed=12)
    gaps = []
    for p in (6, 12):
        s = O.System(pos, q, 6.0, 3, p)
        s.setup()
        rng = np.random.default_rng(13)
        g = 0.0
        for _ in range(6):
            j = int(rng.integers(len(q)))
            r0 = s.positions()[j].copy()
            rn = (r0 + rng.uniform(-0.4, 0.4, 3)) % 6.0
            d1 = s.propose(j, rn)
            s.accept(j, rn, d1)
            g = max(g, abs(d1 + s.propose(j, r0)))
        gaps.append(g)
    assert gaps[1] < gaps[0] and gaps[1] < 1e-5


def test_setup_equals_incremental_accepts():
    """Alg. L.2 adds and removes exactly the P2L terms of Alg. L.3, so after
    accepted moves the expansions equal a fresh setup to roundoff."""
    pos, q = uniform_system(128, 8.0, seed=14)
    a, L, p = 8.0, 3, 8
    s = O.System(pos, q, a, L, p)
    s.setup()
    rng = np.random.default_rng(15)
    for _ in range(25):
        j = int(rng.integers(len(q)))
        rn = (s.positions()[j] + rng.uniform(-1.2, 1.2, 3)) % a
        s.accept(j, rn, s.propose(j, rn))
    f = O.System(s.positions(), q, a, L, p)
    f.setup()
    for lev in range(2, L + 1):
        A, B = s.local(lev), f.local(lev)
        assert np.max(np.abs(A - B)) <= 1e-12 * np.max(np.abs(B))
    Ka, Ha = s.KH()
    Kb, Hb = f.KH()
    assert np.max(np.abs(Ka - Kb)) <= 1e-12 * np.max(np.abs(Kb))
    # running energy equals the fresh energy to truncation level
    assert abs(s.energy() - f.energy()) < 1e-4 * abs(f.energy())


def test_running_energy_tracks_fresh_energy_at_high_order():
    pos, q = uniform_system(64, 5.0, seed=16)
    s = O.System(pos, q, 5.0, 3, 18)
    s.setup()
    res = s.run(300, seed=3, half_width=0.4)
    assert res["n_acc"] > 50
    assert abs(s.energy() - s.energy_fresh()) < 1e-6 * abs(s.energy_fresh())
    Ue = O.ewald_energy(s.positions(), q, 5.0)
    assert abs(s.energy() - Ue) < 1e-5 * abs(Ue)


# ------------------------------------------------------------- MH driver
def test_metropolis_rule_limits():
    pos, q = uniform_system(64, 6.0, seed=17)
    s = O.System(pos, q, 6.0, 3, 4)
    s.setup()
    r = s.run(200, seed=1, beta=0.0, half_width=0.3)
    assert r["n_acc"] == 200
    s2 = O.System(pos, q, 6.0, 3, 4)
    s2.setup()
    r2 = s2.run(200, seed=1, beta=1e12, half_width=0.3)
    assert np.array_equal(r2["acc"].astype(bool), r2["dE"] <= 0)


def test_follow_driver_reproduces_the_chain_and_a_frozen_system():
    """The driver option that takes another chain's decisions: following the
    chain's own decisions gives the chain itself; following "reject all"
    leaves the system as it was, so every dE is a proposal on the initial
    state (Alg. L.1 evaluated directly) and the positions do not move."""
    pos, q = uniform_system(120, 6.0, seed=8)
    a = O.System(pos, q, 6.0, 3, 5)
    a.setup()
    ra = a.run(300, seed=4, step0=10, chain=2, beta=1.0, half_width=0.5)
    b = O.System(pos, q, 6.0, 3, 5)
    b.setup()
    rb = b.run_follow(ra["acc"], seed=4, step0=10, chain=2, beta=1.0, half_width=0.5)
    assert np.array_equal(ra["j"], rb["j"]) and np.array_equal(ra["acc"], rb["acc"])
    assert np.array_equal(ra["dE"], rb["dE"]) and ra["n_acc"] == rb["n_acc"]
    assert np.array_equal(a.positions(), b.positions())
    c = O.System(pos, q, 6.0, 3, 5)
    c.setup()
    rc = c.run_follow(np.zeros(40, np.uint8), seed=4, step0=10, chain=2, beta=1.0, half_width=0.5)
    assert rc["n_acc"] == 0 and np.array_equal(c.positions(), pos)
    d = O.System(pos, q, 6.0, 3, 5)
    d.setup()
    for t in range(40):
        j, dl, _ = O.proposal(120, 0.5, 4, 10 + t, 2)
        rn = (pos[j] + dl) % 6.0
        assert rc["j"][t] == j
        assert rc["dE"][t] == d.propose(j, rn)


def test_proposal_stream_statistics():
    n = 1000
    js, ds, us = [], [], []
    for t in range(20000):
        j, d, u = O.proposal(n, 0.5, seed=7, step=t)
        js.append(j)
        ds.append(d)
        us.append(u)
    js, ds, us = np.array(js), np.array(ds), np.array(us)
    assert js.min() >= 0 and js.max() < n
    counts = np.bincount(js // 100, minlength=10)
    chi2 = ((counts - 2000) ** 2 / 2000).sum()
    assert chi2 < 30  # 9 dof
    assert np.all(np.abs(ds) < 0.5) and abs(ds.mean()) < 0.01
    assert np.all((us >= 0) & (us < 1)) and abs(us.mean() - 0.5) < 0.01
    # distinct counters and chains give distinct blocks
    a = O.philox([1, 0, 0, 0], [7, 0])
    b = O.philox([1, 0, 1, 0], [7, 0])
    c = O.philox([1, 0, 0, 0], [8, 0])
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def test_philox_known_answers():
    """The proposal stream's generator is Philox4x32-10 (Salmon et al.,
    SC'11): the oracle's implementation reproduces the published
    known-answer values (tests/golden/philox_kat.txt)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = O.philox(w[0:4], w[4:6])
        assert [int(v) for v in out] == w[6:10], r


def test_fmm_variant_setup_converges_to_exact_setup_and_direct_sums():
    """The FMM-variant setup (Sec. 3.2: per-level multipoles translated into
    each cell's interaction list) equals Alg. L.3 up to the multipole
    truncation, so its distance to the P2L setup falls with p; in free space
    its energy converges to the direct pair sum."""
    pos, q = uniform_system(200, 6.0, seed=21)
    gaps = []
    for p in (4, 6, 8):
        a = O.System(pos, q, 6.0, 3, p)
        a.setup()
        b = O.System(pos, q, 6.0, 3, p)
        b.setup_fmm()
        gaps.append(max(np.max(np.abs(a.local(l) - b.local(l))) / np.max(np.abs(a.local(l)))
                        for l in (2, 3)))
        Ka, _ = a.KH()
        Kb, _ = b.KH()
        assert np.max(np.abs(Ka - Kb)) <= 1e-12 * np.max(np.abs(Ka))
    assert gaps[0] > 3 * gaps[1] > 9 * gaps[2] and gaps[2] < 5e-5
    pos, q = uniform_system(200, 8.0, seed=22)
    Ud = O.direct_energy(pos, q)
    errs = []
    for p in (4, 8, 12):
        b = O.System(pos, q, 8.0, 3, p, bc=O.BC_FREE)
        b.setup_fmm()
        errs.append(abs(b.energy() - Ud) / abs(Ud))
    assert errs[0] > 10 * errs[1] > 100 * errs[2] and errs[2] < 1e-6


# ------------------------------------------------ multipole method (Alg. M)
def test_multipole_method_energy_and_moves_match_ewald():
    """Alg. M.3/M.1 with the periodic terms: the energy converges to Ewald
    geometrically in p and dE of (wrapped) moves matches Ewald differences."""
    pos, q = uniform_system(32, 4.0, seed=5)
    a = 4.0
    Ue = O.ewald_energy(pos, q, a)
    errs = []
    for p in (8, 14, 20):
        s = O.System(pos, q, a, 3, p)
        s.setup_multipole()
        errs.append(abs(s.energy() - Ue))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-6 * abs(Ue)
    s = O.System(pos, q, a, 3, 20)
    s.setup_multipole()
    rng = np.random.default_rng(7)
    for _ in range(5):
        j = int(rng.integers(len(q)))
        rn = (pos[j] + rng.uniform(-0.8, 0.8, 3)) % a
        dE = s.propose(j, rn)
        pos2 = pos.copy()
        pos2[j] = rn
        dEx = O.ewald_energy(pos2, q, a) - O.ewald_energy(pos, q, a)
        assert abs(dE - dEx) < 1e-6 * max(1.0, abs(dEx))
        s.accept(j, rn, dE)
        pos = pos2


def test_multipole_method_free_space_matches_direct_sums():
    pos, q = uniform_system(48, 8.0, seed=8)
    s = O.System(pos, q, 8.0, 4, 20, bc=O.BC_FREE)
    s.setup_multipole()
    Ud = O.direct_energy(pos, q)
    assert abs(s.energy() - Ud) < 1e-7 * abs(Ud)
    rng = np.random.default_rng(9)
    for _ in range(5):
        j = int(rng.integers(len(q)))
        rn = np.clip(pos[j] + rng.uniform(-1.5, 1.5, 3), 0.0, 7.999)
        dE = s.propose(j, rn)
        pos2 = pos.copy()
        pos2[j] = rn
        dEx = O.direct_energy(pos2, q) - Ud
        assert abs(dE - dEx) < 1e-7 * max(1.0, abs(dEx))
        s.accept(j, rn, dE)
        pos, Ud = pos2, Ud + dEx


def test_multipole_method_accepts_equal_fresh_setup_and_track_local_method():
    """Alg. M.2 adds and removes exactly the terms of Alg. M.3; the
    multipole and local methods approximate the same dE, so their gap falls
    with p."""
    pos, q = uniform_system(128, 8.0, seed=14)
    a, L = 8.0, 3
    s = O.System(pos, q, a, L, 8)
    s.setup_multipole()
    rng = np.random.default_rng(15)
    for _ in range(25):
        j = int(rng.integers(len(q)))
        rn = (s.positions()[j] + rng.uniform(-1.2, 1.2, 3)) % a
        s.accept(j, rn, s.propose(j, rn))
    f = O.System(s.positions(), q, a, L, 8)
    f.setup_multipole()
    for lev in range(2, L + 1):
        A, B = s.multipole(lev), f.multipole(lev)
        assert np.max(np.abs(A - B)) <= 1e-12 * np.max(np.abs(B))
    gaps = []
    for p in (6, 12):
        m = O.System(pos, q, a, L, p)
        m.setup_multipole()
        loc = O.System(pos, q, a, L, p)
        loc.setup()
        rng = np.random.default_rng(16)
        g = 0.0
        for _ in range(6):
            j = int(rng.integers(len(q)))
            rn = (pos[j] + rng.uniform(-0.5, 0.5, 3)) % a
            g = max(g, abs(m.propose(j, rn) - loc.propose(j, rn)))
        gaps.append(g)
    assert gaps[1] < 0.1 * gaps[0] and gaps[1] < 1e-4


# ------------------------------------------- short-range Lennard-Jones term
def _lj_brute(pos, a, eps, sig, rc, skip=None):
    """all pairs, minimum image (a >= 2 rc, so at most one image is in range)"""
    u = 0.0
    n = len(pos)
    for i in range(n):
        for k in range(i + 1, n):
            d = pos[i] - pos[k]
            d -= a * np.round(d / a)
            r = np.linalg.norm(d)
            if r < rc:
                u += 4 * eps * ((sig / r) ** 12 - (sig / r) ** 6)
    return u


def test_lennard_jones_energy_and_moves_match_pair_sums():
    """The LJ term of Sec. 5.3 (cutoff no larger than the finest cell, so
    the 27 near cells hold every pair in range): energy and dE equal direct
    minimum-image pair sums; the moving particle's old copy is excluded."""
    a, L, rc, eps, sig = 24.0, 2, 12.0, 0.02, 1.1
    pos, q = uniform_system(60, a, seed=41)
    base = O.System(pos, q, a, L, 8)
    base.setup()
    s = O.System(pos, q, a, L, 8)
    s.set_lj(eps, sig, rc)
    s.setup()
    assert abs((s.energy() - base.energy()) - _lj_brute(pos, a, eps, sig, rc)) < 1e-10
    rng = np.random.default_rng(42)
    for _ in range(4):
        j = int(rng.integers(len(q)))
        rn = (pos[j] + rng.uniform(-0.4, 0.4, 3)) % a
        pos2 = pos.copy()
        pos2[j] = rn
        dlj = _lj_brute(pos2, a, eps, sig, rc) - _lj_brute(pos, a, eps, sig, rc)
        assert abs((s.propose(j, rn) - base.propose(j, rn)) - dlj) < 1e-10
    with pytest.raises(ValueError):
        s.set_lj(eps, sig, 12.5)  # beyond the finest cell width


@pytest.mark.parametrize("bc", [O.BC_PBC, O.BC_FREE])
def test_local_cell_direct_equals_the_setup(bc):
    """Alg. L.3 for one cell by its definition (gathered from the charges of
    its interaction list, no setup) equals the cell of the full setup
    (scattered particle by particle), on every level: the two are the same
    sum in another order, through the symmetry of the interaction list."""
    n, a, L, p = 700, 9.0, 4, 7
    pos, q = uniform_system(n, a, seed=31)
    o = O.System(pos, q, a, L, p, bc=bc)
    d = O.System(pos, q, a, L, p, bc=bc)  # never set up
    o.setup()
    rng = np.random.default_rng(5)
    for lev in range(2, L + 1):
        nl = 1 << (lev - 1)
        full = o.local(lev)
        scale = np.max(np.abs(full))
        cells = [np.array(c) for c in np.ndindex(nl, nl, nl)] if nl <= 4 else \
            [rng.integers(0, nl, size=3) for _ in range(12)]
        for c in cells:
            got = d.local_cell_direct(lev, c)
            ref = full[(c[0] * nl + c[1]) * nl + c[2]]
            assert np.max(np.abs(got - ref)) <= 1e-13 * scale, (lev, c)
    with pytest.raises(ValueError):
        d.local_cell_direct(1, [0, 0, 0])
    with pytest.raises(ValueError):
        d.local_cell_direct(L, [1 << (L - 1), 0, 0])
