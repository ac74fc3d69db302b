"""CPU checks of the matvec pass planner and the complex64 record layout.

The H psi kernel applies the Pauli strings of a block pass by pass (each pass
visits super-tiles: the amplitudes sharing one value of the index bits its
covered terms never flip) and reads them as packed records ordered into runs
of equal input tile.  None of this may change the product (Algorithm 1 is a
plain sum over terms), so these tests check, without a GPU, that

* the plan is a partition of the compiled terms, in the documented order;
* every covered term stays inside its pass's super-tile, the super-tile fits
  the budget, and the tile visit order is a permutation that walks one
  super-tile at a time;
* the records carry exactly the plan's terms, runs, flags and sign bits, and
  H psi evaluated from the records alone equals the oracle's block
  Hamiltonian applied to psi (to the records' float32 coefficient rounding);
* split passes cover their terms with non-empty chunks;
* the same holds for the compiled string tables of spin chains and of
  complex couplings (syk_plan_strings_host), and the benchmark's L=31 chain
  gets the plan its ncu summary describes.
"""
import os

import numpy as np
import pytest

import syk_inputs as si
from oracle import hamiltonian as ham

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TILE_BITS = 11
MASK31 = np.uint32(0x7FFFFFFF)


@pytest.fixture(scope="module")
def pkg():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_syk_build", os.path.join(ROOT, "paper_2311_00639_b300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_2311_00639_b300 as p

    return p


def term_class(x, z, imag):
    return 4 * imag.astype(np.int64) + 2 * (x & 1).astype(np.int64) + (z & 1).astype(np.int64)


def tile_starts(p, nh):
    b = np.arange(1 << nh, dtype=np.int64)
    dep = p["dep"].astype(np.int64)
    return dep[0][b & 255] | dep[1][(b >> 8) & 255] | dep[2][(b >> 16) & 255]


def unpack(rec):
    """records [n + 1][4] -> x, z, coef, flags (x and z with bit 31 cleared)."""
    return rec[:, 0] & MASK31, rec[:, 1] & MASK31, rec[:, 2].view(np.float32).astype(np.float64), rec[:, 3]


# (N, k, dtype, budget, ratio): default plans, tight budgets that force several
# passes at small sizes, the straggler rule on and off
CASES = [
    (26, 4, "c64", 4096, 0.0),
    (28, 4, "c64", 8192, 3.0),
    (30, 8, "c64", 16384, 0.0),
    (30, 8, "c64", 16384, 1.5),
    (32, 4, "c128", 32768, 1.5),
    (34, 2, "c64", 0, 0.0),
    (64, 4, "c64", 0, 0.0),
    (64, 4, "c128", 0, 0.0),
]


@pytest.mark.parametrize("N,k,dtype,budget,ratio", CASES)
def test_plan_partitions_terms_in_order(pkg, N, k, dtype, budget, ratio):
    q, J, _ = si.sample_sparse_syk(N, k, r=N)
    plan = pkg.plan_host(N, q, J, dtype, "jw", budget, ratio)
    ref = pkg.compile_terms_host(N, q, J, "jw")
    n = len(ref["x"])
    assert len(plan["x"]) == n
    key = lambda d: sorted(zip(d["x"].tolist(), d["z"].tolist(), d["coef_U"].tolist(), d["coef_D"].tolist(),
                               d["imag"].tolist()))
    assert key(plan) == key(ref)  # the same strings, only reordered
    passes = plan["passes"]
    assert passes[0]["t0"] == 0 and passes[-1]["t1"] == n
    cls = term_class(plan["x"], plan["z"], plan["imag"])
    for a, b in zip(passes, passes[1:]):
        assert a["t1"] == b["t0"] and a["t1"] > a["t0"]
    for p in passes:
        c = p["cls"]
        assert c[0] == p["t0"] and c[8] == p["t1"] and c[4] == p["ti"]
        assert all(c[i] <= c[i + 1] for i in range(8))
        for ci in range(8):
            assert np.all(cls[c[ci]:c[ci + 1]] == ci)
        seg = list(zip(cls[p["t0"]:p["t1"]].tolist(), plan["x"][p["t0"]:p["t1"]].tolist(),
                       plan["z"][p["t0"]:p["t1"]].tolist()))
        assert seg == sorted(seg)
    if budget and ratio == 0.0:  # budget 0 takes the default ratio too
        assert not plan["straggler"].any()


@pytest.mark.parametrize("N,k,dtype,budget,ratio", CASES)
def test_super_tiles_fit_budget_and_hold_covered_terms(pkg, N, k, dtype, budget, ratio):
    q, J, _ = si.sample_sparse_syk(N, k, r=N)
    plan = pkg.plan_host(N, q, J, dtype, "jw", budget, ratio)
    L = N // 2 - 1
    nh = max(0, L - TILE_BITS)
    elem = 8 if dtype == "c64" else 16
    if budget == 0:
        budget = (32 << 20) if dtype == "c64" else (2 << 20)
    vec = (1 << L) * elem
    e = 0
    while e < nh and (vec >> e) > budget:
        e += 1
    for p in plan["passes"]:
        em = p["emask"]
        assert em & ((1 << TILE_BITS) - 1) == 0 and em < (1 << L)
        assert bin(em).count("1") in (0, e)
        if bin(em).count("1") == e and e > 0:
            # the fewest fixed bits whose super-tile fits (all high bits if none fits)
            assert ((vec >> e) <= budget or e == nh) and budget < (vec >> (e - 1))
        sl = slice(p["t0"], p["t1"])
        covered = plan["straggler"][sl] == 0
        assert np.all((plan["x"][sl][covered] & np.uint32(em)) == 0)
        # tile visit order: a permutation of the tiles, one super-tile after another
        starts = tile_starts(p, nh)
        assert np.array_equal(np.sort(starts), np.arange(1 << nh, dtype=np.int64) << TILE_BITS)
        G = 1 << (nh - bin(em).count("1"))
        groups = starts.reshape(-1, G)
        assert np.all((groups & em) == (groups[:, :1] & em))
        # a covered term maps each super-tile onto itself
        for x in np.unique(plan["x"][sl][covered] & ~np.uint32((1 << TILE_BITS) - 1)):
            g0 = np.sort(groups[0])
            assert np.array_equal(np.sort(g0 ^ int(x)), g0)


@pytest.mark.parametrize("N,k,dtype,budget,ratio", CASES)
def test_records_runs_flags_and_sign_bits(pkg, N, k, dtype, budget, ratio):
    q, J, _ = si.sample_sparse_syk(N, k, r=N)
    plan = pkg.plan_host(N, q, J, dtype, "jw", budget, ratio)
    n = len(plan["x"])
    R = plan["records"]
    assert np.all(R[:, n] == 0)  # the zero record past the end
    n_runs = 0
    for blk, coef in ((0, plan["coef_U"]), (1, plan["coef_D"])):
        x, z, c, fl = unpack(R[blk, :n])
        # raw bit 31 of flags, x, z = z bits 6, 7, 8
        assert np.array_equal(R[blk, :n, 3] >> 31, (z >> 6) & 1)
        assert np.array_equal(R[blk, :n, 0] >> 31, (z >> 7) & 1)
        assert np.array_equal(R[blk, :n, 1] >> 31, (z >> 8) & 1)
        imag = (fl >> 3) & 1
        body = (fl >> 8) & 63
        assert np.array_equal(body, 32 * imag + 16 * (x & 1) + 8 * (z & 1) + ((x >> 6) & 7))
        assert np.all(fl & np.uint32(0x7F00C0E0) == 0)  # no stray bits
        n_runs_blk = n_merges_blk = 0
        for p in plan["passes"]:
            sl = slice(p["t0"], p["t1"])
            # same terms as the plan's pass, as a multiset
            got = sorted(zip(x[sl].tolist(), z[sl].tolist(), c[sl].tolist(), imag[sl].tolist(),
                             (fl[sl] & 1).tolist()))
            want = sorted(zip(plan["x"][sl].tolist(), plan["z"][sl].tolist(),
                              coef[sl].astype(np.float32).astype(np.float64).tolist(),
                              plan["imag"][sl].astype(np.uint32).tolist(),
                              plan["straggler"][sl].astype(np.uint32).tolist()))
            assert got == want
            # ordered by (input tile, class, x, z); runs = maximal equal-tile stretches
            hi = x[sl] >> TILE_BITS
            key = list(zip(hi.tolist(), term_class(x[sl], z[sl], imag[sl]).tolist(), x[sl].tolist(),
                           z[sl].tolist()))
            assert key == sorted(key)
            start = np.r_[True, hi[1:] != hi[:-1]]
            end = np.r_[hi[1:] != hi[:-1], True]
            assert np.array_equal((fl[sl] >> 1) & 1, start.astype(np.uint32))
            assert np.array_equal((fl[sl] >> 2) & 1, end.astype(np.uint32))
            n_runs_blk += int(start.sum())
            assert int(start.sum()) == len(np.unique(hi))
            # merge groups: stretches of equal x and class, in groups of at most 256 records;
            # merge flag = the next record is in the same group, bits 16-23 of a group's first
            # record = the records after it
            cl = term_class(x[sl], z[sl], imag[sl])
            same = np.r_[(x[sl][1:] == x[sl][:-1]) & (cl[1:] == cl[:-1]), False]
            merge = np.zeros(len(same), bool)
            glen = np.zeros(len(same), np.uint32)
            i = 0
            while i < len(same):
                e = i
                while same[e]:
                    e += 1
                for a in range(i, e + 1, 256):
                    b = min(e, a + 255)
                    glen[a] = b - a
                    merge[a:b] = True
                i = e + 1
            assert np.array_equal((fl[sl] >> 4) & 1, merge.astype(np.uint32))
            assert np.array_equal((fl[sl] >> 16) & 255, glen)
            n_merges_blk += int(merge.sum())
        n_runs = n_runs_blk
        assert plan["n_merges"] == n_merges_blk
    assert plan["n_runs"] == n_runs


@pytest.mark.parametrize("N,k,budget,ratio,rep", [(26, 4, 4096, 0.0, "jw"), (28, 6, 8192, 3.0, "jw"),
                                                 (28, 4, 8192, 1.5, "paper")])
def test_records_alone_reproduce_oracle_block(pkg, N, k, budget, ratio, rep):
    """H_P psi from the records only (masked x and z, float32 coefficient, imag
    flag) against the oracle's CSR block, term rounding bound 2^-24 sum |c|."""
    q, J, _ = si.sample_sparse_syk(N, k, r=N + 1)
    plan = pkg.plan_host(N, q, J, "c64", rep, budget, ratio)
    assert len(plan["passes"]) >= 2
    n = len(plan["x"])
    D = 1 << (N // 2 - 1)
    rng = np.random.default_rng(N)
    psi = rng.normal(size=D) + 1j * rng.normal(size=D)
    m = np.arange(D, dtype=np.int64)
    for blk in (0, 1):
        x, z, c, fl = unpack(plan["records"][blk, :n])
        out = np.zeros(D, dtype=np.complex128)
        for xt, zt, ct, ft in zip(x.tolist(), z.tolist(), c.tolist(), fl.tolist()):
            sign = 1.0 - 2.0 * (np.bitwise_count(m & zt) & 1)
            out += (1j * ct if (ft >> 3) & 1 else ct) * sign * psi[m ^ xt]
        ref = ham.csr_block(N, q, J, rep, blk) @ psi
        bound = 2.0 ** -24 * np.abs(c).sum() * np.abs(psi).max() * 1.01 + 1e-12
        assert np.max(np.abs(out - ref)) <= bound


def test_split_plan_covers_terms(pkg):
    # small blocks (few tiles) with many terms per pass are split across CTAs
    for N, dtype, n_sm in [(30, "c64", 148), (32, "c64", 148), (30, "c64", 4), (30, "c128", 148), (40, "c64", 148)]:
        q, J = si.sample_dense_syk(N, seed=1)[:2] if N <= 30 else si.sample_sparse_syk(N, 16, r=1)[:2]
        plan = pkg.plan_host(N, q, J, dtype, "jw", 0, 0.0, n_sm)
        D = 1 << (N // 2 - 1)
        ntiles = D >> TILE_BITS
        # resident CTAs of the store passes: 4 per SM when the handle's runs are long (16 or more
        # terms per staged tile) or half of its terms merge, else 5
        n_terms = len(plan["x"])
        wide = 2 * plan["n_merges"] >= n_terms > 0 and plan["n_merges"] > 0 or n_terms >= 16 * max(plan["n_runs"], 1)
        cap = n_sm * (4 if wide else 5)
        any_split = False
        for p in plan["passes"]:
            Tp, C, Tc = p["t1"] - p["t0"], p["split_chunks"], p["split_terms"]
            if dtype == "c128" or 2 * ntiles > cap or Tp < 64:
                assert C == 1 and Tc == 0
                continue
            any_split = True
            assert C >= 2 and Tc >= 32 and (C - 1) * Tc < Tp <= C * Tc  # every chunk non-empty
            assert C == -(-Tp // -(-Tp // min(-(-cap // ntiles), Tp // 32)))  # plan_split's chunk count
        assert any_split == (dtype == "c64" and 2 * ntiles <= cap and any(
            p["t1"] - p["t0"] >= 64 for p in plan["passes"]))


def test_default_N64_plan(pkg):
    """The default complex64 plan of the N=64, k=4 workload (T=261 strings):
    7 passes of 102, 64, 34, 26, 15, 11, 9 terms, 12 of them stragglers, and
    218 input tiles staged per output tile."""
    q, J, _ = si.sample_sparse_syk(64, 4, r=0)
    plan = pkg.plan_host(64, q, J, "c64")
    assert [p["t1"] - p["t0"] for p in plan["passes"]] == [102, 64, 34, 26, 15, 11, 9]
    assert int(plan["straggler"].sum()) == 12 and plan["n_runs"] == 218
    # deterministic: the same input gives the same plan
    again = pkg.plan_host(64, q, J, "c64")
    assert np.array_equal(again["records"], plan["records"])


def test_plan_host_rejects_bad_arguments(pkg):
    from paper_2311_00639_b300 import SykError

    q, J, _ = si.sample_sparse_syk(20, 4, r=0)
    with pytest.raises(SykError):
        pkg.plan_host(20, q, J, "c64", "jw", 100, 1.0)
    with pytest.raises(SykError):
        pkg.plan_host(20, q, J, "c64", "jw", 0, -1.0)
    with pytest.raises(SykError):
        pkg.plan_host(20, q, J, "c64", "jw", 0, 0.0, 0)
    empty = pkg.plan_host(20, np.zeros((0, 4), np.int32), np.zeros(0), "c64")
    assert len(empty["x"]) == 0 and len(empty["passes"]) == 1 and empty["n_runs"] == 0


def _records_apply(records, n, psi):
    """H psi from one block's records alone (masked masks, float32 coefficient, imag flag)."""
    D = len(psi)
    m = np.arange(D, dtype=np.int64)
    x, z, c, fl = unpack(records[:n])
    out = np.zeros(D, dtype=np.complex128)
    for xt, zt, ct, ft in zip(x.tolist(), z.tolist(), c.tolist(), fl.tolist()):
        sign = 1.0 - 2.0 * (np.bitwise_count(m & zt) & 1)
        out += (1j * ct if (ft >> 3) & 1 else ct) * sign * psi[m ^ xt]
    return out, np.abs(c).sum()


@pytest.mark.parametrize("L,budget,ratio", [(16, 1 << 14, 0.0), (16, 1 << 15, 3.0), (14, 0, 0.0)])
def test_plan_strings_spin_chain_records_reproduce_oracle(pkg, L, budget, ratio):
    """The host plan view of a Pauli-string table (syk_plan_strings_host): a
    partition of the compiled strings, and records that alone apply the
    oracle's spin Hamiltonian."""
    from oracle import spin

    x, z, h, _ = si.heisenberg_chain(L, W=2.0, r=7)
    x2, z2, h2 = si.random_pauli_terms(L, 30, seed=9, max_weight=4)
    x, z, h = np.concatenate([x, x2]), np.concatenate([z, z2]), np.concatenate([h, h2])
    comp = pkg.compile_pauli_host(L, x, z, h)
    plan = pkg.plan_strings_host(L, comp, "c64", budget, ratio)
    n = len(comp["x"])
    key = lambda xs, zs, cs, ims: sorted(zip(xs.tolist(), zs.tolist(), cs.tolist(), ims.tolist()))
    assert key(plan["x"], plan["z"], plan["coef_U"], plan["imag"]) == key(comp["x"], comp["z"], comp["coef"],
                                                                         comp["imag"])
    assert np.array_equal(plan["coef_U"], plan["coef_D"])
    if budget:
        assert len(plan["passes"]) >= 2
    psi = np.random.default_rng(L).normal(size=1 << L) + 0j
    ref = spin.csr_H(L, x, z, h) @ psi
    for blk in (0, 1):
        out, s = _records_apply(plan["records"][blk], n, psi)
        assert np.max(np.abs(out - ref)) <= 2.0 ** -24 * s * np.abs(psi).max() * 1.01 + 1e-12


def test_plan_strings_complex_couplings_records_reproduce_oracle(pkg):
    """Non-Hermitian SYK (complex couplings): real- and imaginary-class strings
    with equal masks share runs; the records alone apply the oracle's blocks."""
    from oracle import nonherm as nh

    N = 28
    q, J, _ = si.sample_sparse_syk(N, 4, r=5)
    M = np.random.default_rng(5).normal(size=len(J)) * np.sqrt(np.mean(J ** 2))
    comp = pkg.compile_terms_complex_host(N, q, J, M, "jw")
    plan = pkg.plan_strings_host(N // 2 - 1, comp, "c64", 8192, 3.0)
    n = len(comp["x"])
    assert n == 2 * len(J)  # every term: a real and an imaginary string
    assert plan["n_runs"] <= len(np.unique(comp["x"] >> TILE_BITS)) * len(plan["passes"])
    psi = np.random.default_rng(1).normal(size=1 << (N // 2 - 1)) + 1j
    for blk in (0, 1):
        out, s = _records_apply(plan["records"][blk], n, psi)
        ref = nh.csr_block(N, q, J, M, "jw", blk) @ psi
        assert np.max(np.abs(out - ref)) <= 2.0 ** -24 * s * np.abs(psi).max() * 1.01 + 1e-12


def test_default_heisenberg_L31_plan(pkg):
    """The default complex64 plan of the benchmark's chain (L=31, W=5, 124
    strings): 2 passes of 104 and 20 strings, 12 + 10 staged tiles per output
    tile, as in the ncu summary of that workload."""
    x, z, h, _ = si.heisenberg_chain(31, 5.0, r=0)
    plan = pkg.plan_strings_host(31, pkg.compile_pauli_host(31, x, z, h), "c64")
    assert [p["t1"] - p["t0"] for p in plan["passes"]] == [104, 20]
    assert plan["n_runs"] == 22 and not plan["straggler"].any()


def test_plan_strings_rejects_bad_arguments(pkg):
    from paper_2311_00639_b300 import SykError

    comp = {"x": np.array([1 << 5], np.uint32), "z": np.zeros(1, np.uint32), "coef": np.ones(1),
            "imag": np.zeros(1, np.uint8)}
    with pytest.raises(SykError):
        pkg.plan_strings_host(5, comp)  # bit 5 of a 5-bit index
    with pytest.raises(SykError):
        pkg.plan_strings_host(0, comp)
    comp["x"][0] = 1
    assert len(pkg.plan_strings_host(5, comp)["x"]) == 1


def test_merge_groups_of_dense_records_reproduce_oracle_block(pkg):
    """Dense SYK (every quadruple): many strings share a flip mask. Records
    flagged "merge" (bit 4) form groups of equal x and class, which the
    complex64 kernel applies once with the summed signed coefficients. Summing
    each group's coefficients first and applying one permutation per group
    reproduces the oracle's block."""
    N = 16
    q, J, _ = si.sample_dense_syk(N, seed=2)
    plan = pkg.plan_host(N, q, J, "c64", "jw", 0, 0.0, 148)
    n = len(plan["x"])
    assert plan["n_merges"] > n // 2  # most terms merge at this size
    D = 1 << (N // 2 - 1)
    rng = np.random.default_rng(3)
    psi = rng.normal(size=D) + 1j * rng.normal(size=D)
    m = np.arange(D, dtype=np.int64)
    for blk in (0, 1):
        x, z, c, fl = unpack(plan["records"][blk, :n])
        out = np.zeros(D, dtype=np.complex128)
        acc = np.zeros(D)
        groups = 0
        for k in range(n):
            sign = 1.0 - 2.0 * (np.bitwise_count(m & int(z[k])) & 1)
            acc = acc + c[k] * sign
            if (fl[k] >> 4) & 1:
                assert x[k + 1] == x[k] and ((fl[k + 1] >> 3) & 1) == ((fl[k] >> 3) & 1)
                continue
            out += (1j if (fl[k] >> 3) & 1 else 1.0) * acc * psi[m ^ int(x[k])]
            acc = np.zeros(D)
            groups += 1
        assert groups == n - plan["n_merges"]
        ref = ham.csr_block(N, q, J, "jw", blk) @ psi
        bound = 2.0 ** -24 * np.abs(c).sum() * np.abs(psi).max() * 1.01 + 1e-12
        assert np.max(np.abs(out - ref)) <= bound


def test_long_stretches_split_into_merge_groups_of_256(pkg):
    """600 strings with one flip mask and class: merge groups of 256, 256 and
    88 records (bits 16-23 of each group's first record: 255, 255, 87); the
    records alone, summing each group first, reproduce the oracle's block."""
    from oracle import spin

    L, n = 12, 600
    rng = np.random.default_rng(7)
    z = rng.choice(np.arange(2, 1 << L, 2), size=n, replace=False).astype(np.uint32)
    x, h = np.zeros(n, np.uint32), rng.normal(size=n)
    comp = pkg.compile_pauli_host(L, x, z, h)
    plan = pkg.plan_strings_host(L, comp, "c64", 0, 0.0, 148)
    R = plan["records"][0, :n]
    fl = R[:, 3]
    starts = np.nonzero((fl >> 16) & 255)[0]
    assert ((fl[starts] >> 16) & 255).tolist() == [255, 255, 87]
    assert starts.tolist() == [0, 256, 512]
    assert int(((fl >> 4) & 1).sum()) == plan["n_merges"] == n - 3
    D = 1 << L
    psi = rng.normal(size=D) + 1j * rng.normal(size=D)
    m = np.arange(D, dtype=np.int64)
    out = np.zeros(D, dtype=np.complex128)
    xr, zr, c, _ = unpack(R)
    for a, g in zip(starts.tolist(), ((fl[starts] >> 16) & 255).tolist()):
        acc = np.zeros(D)
        for k in range(a, a + g + 1):
            acc += c[k] * (1.0 - 2.0 * (np.bitwise_count(m & int(zr[k])) & 1))
        out += acc * psi[m ^ int(xr[a])]
    ref = spin.csr_H(L, x, z, h) @ psi
    assert np.max(np.abs(out - ref)) <= 2.0 ** -24 * np.abs(c).sum() * np.abs(psi).max() * 1.01 + 1e-12
