"""Host-side checks of the C ABI (no GPU): the library loads, exports every entry point
declared in include/mpps.h, and its precision planner agrees exactly with the oracle's
statement of the rule (eq. (2.8), Algorithm 3.1 / 4.1, Section 4.1.1)."""
import os
import re

import math

import numpy as np
import pytest

import oracle
from conftest import ROOT


@pytest.fixture(scope="module")
def mpps():
    from paper_2312_17396_gb300 import _build
    _build.build()
    import paper_2312_17396_gb300 as m
    m.lib()
    return m


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mpps.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?\s*([A-Za-z_][A-Za-z_0-9]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "for", "sizeof")))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("ps_eval", "expm_taylor_ss", "ps_eval_adjoint", "mpps_plan", "mpps_matmul",
                 "mpps_last_error", "mpps_version", "mpps_policy_default"):
        assert must in names


def test_library_exports_every_declared_symbol(mpps):
    L = mpps.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert "sm_103a" in mpps.version()


def test_library_binding_lists_all_exports(mpps):
    assert set(declared_functions()) <= set(mpps.EXPORTS)


def test_invalid_arguments_rejected_without_gpu(mpps):
    with pytest.raises(mpps.MppsError) as e:
        mpps.plan(-1, 4, [1.0], 1.0)
    assert e.value.status == 1
    with pytest.raises(mpps.MppsError):
        mpps.plan(16, 0, [1.0] * 5, 1.0)
    # the products reject a bad format or a null matrix before any GPU work, and do nothing
    # for an empty batch
    L = mpps.lib()
    for f in (L.mpps_matmul, L.mpps_matmul_ta):
        assert f(None, None, None, 8, 1, 7, None) == 1
        assert f(None, None, None, 8, 1, 0, None) == 1
        assert f(None, None, None, 0, 1, 0, None) == 1
        assert f(None, None, None, 8, 0, 0, None) == 0
    assert L.mpps_matmul_ta(None, None, None, 8, 1, 7, None) == 1
    assert b"mpps_matmul_ta" in L.mpps_last_error()


def _rand_case(rng):
    m = int(rng.integers(1, 60))
    s = oracle.ceil_sqrt(m)
    r = m // s
    n = int(rng.choice([1, 8, 64, 1024, 4096, 2 ** 20]))
    norms = [float(x) for x in 10.0 ** rng.uniform(-40, 3, size=r + 1)]
    if rng.random() < 0.1:
        norms[int(rng.integers(0, r + 1))] = 0.0
    y = float(10.0 ** rng.uniform(-6, 2))
    return m, n, norms, y


@pytest.mark.parametrize("mode", [oracle.MODE_FIXED, oracle.MODE_PAPER, oracle.MODE_NS])
def test_planner_matches_oracle_rule(mpps, mode):
    rng = np.random.default_rng(7 + mode)
    masks = [0x1F, 0x07, 0x19, 0x01, 0x11]
    for _ in range(400):
        m, n, norms, y = _rand_case(rng)
        mask = int(rng.choice(masks))
        tol = float(rng.choice([2.0 ** -53, 1e-15, 1e-10]))
        k = int(rng.choice([0, 0, 6, 8, 9]))
        ref = oracle.plan(m, n, norms, y, mode=mode, tol=tol, formats=mask, floor_steps=2,
                          f64_slices=k)
        got = mpps.plan(m, n, norms, y, mpps.Policy(mode=mode, tol=tol, formats=mask,
                                                    fp64_floor_steps=2, f64_slices=k))
        assert (got["s"], got["r"], got["nu"], got["fold"]) == \
            (ref["s"], ref["r"], ref["nu"], ref["fold"])
        names = [None] + [mpps.FORMAT_NAMES[f] for f in ref["fmt"][1:]]
        assert got["fmt"] == names
        assert got["u"][1:] == ref["u"][1:]


def test_planner_cost_ratio_reproduces_eq_3_8(mpps):
    # FP64 everywhere -> ratio 1; one product in FP8 -> digits drop by 16 - 1.2
    p = mpps.plan(16, 64, [1.0, 1e-3, 1e-9, 1e-15, 1e-21], 0.5, mpps.Policy(mode=mpps.MIXED_PAPER))
    assert p["fmt"][1:] == ["fp64", "fp64", "fp8", "none"]
    D = -np.log10(2.0 ** -53)
    expect = (3 * D + D + D + (-np.log10(2.0 ** -4)) + 0.0) / ((4 + 4 - 1) * D)
    assert abs(p["cost_ratio"] - expect) < 1e-12
    f = mpps.plan(16, 64, [1.0, 1e-3, 1e-9, 1e-15, 1e-21], 0.5, mpps.FIXED)
    assert abs(f["cost_ratio"] - (3 * D + 3 * D) / (7 * D)) < 1e-12


def test_planner_emulated_ladder(mpps):
    """With emulation (K = 8 slices of 7 bits) the rungs F64E(4..7) sit between BF16X3 and the
    working precision F64E(8): u_i = 1e-9 needs 2^(2-7k) <= 1e-9, i.e. k = 5 (2^-33 = 1.2e-10);
    u_i = 1e-13 needs k = 7 (2^-47 = 7.1e-15)."""
    tol = 2.0 ** -53
    norms = [1.0, tol / 1e-9, tol / 1e-13, 1e-40]          # y = 1 -> u_1 = 1e-9, u_2 = 1e-13
    p = mpps.plan(9, 64, norms, 1.0, mpps.Policy(mode=mpps.MIXED_PAPER, f64_slices=8))
    assert p["fmt"][1:] == ["f64e5", "f64e7", "none"]
    f = mpps.plan(9, 64, norms, 1.0, mpps.Policy(mode=mpps.FIXED_FP64, f64_slices=8))
    assert f["fmt"][1:] == ["f64e8", "f64e8", "none"]
    with pytest.raises(mpps.MppsError):
        mpps.plan(9, 64, norms, 1.0, mpps.Policy(f64_slices=10))


def test_variable_s_rule_matches_oracle(mpps):
    """The library's variable-s rule (Algorithm 3.1, fix_params false) against the oracle's
    statement of it, on random norm sequences around the growth condition."""
    rng = np.random.default_rng(31)
    for _ in range(500):
        m = int(rng.integers(1, 80))
        s0 = oracle.ceil_sqrt(m)
        normX = float(rng.choice([s0 / np.e, s0 / np.e * (1 + 1e-12), 10.0 ** rng.uniform(-3, 0.5)]))
        ln = int(rng.integers(1, 12))
        b0 = 10.0 ** rng.uniform(-2, 1, size=ln)
        # ||Y|| near ||B_0|| ||X||^s, on either side
        y = np.array([b0[k] * normX ** (s0 + k) * 10.0 ** rng.uniform(-1, 1) for k in range(ln)])
        assert mpps.choose_s(m, normX, b0, y) == oracle.choose_s(m, normX, list(b0), list(y))


def test_autotune_table_host_calls(mpps):
    """Switching measured schedule choice on and off and clearing its table need no GPU."""
    mpps.autotune_clear()
    assert mpps.autotune_entries() == []
    mpps.autotune(True)
    mpps.autotune(False)
    mpps.autotune_clear()
    assert mpps.autotune_entries() == []


def test_new_bindings_validate_shapes_before_any_gpu_work(mpps):
    """Shape errors of the Pade, adjoint and variable-s bindings are raised on the host."""
    A = np.zeros((2, 4, 4)); G = np.zeros((2, 5, 5))
    with pytest.raises(ValueError):
        mpps.expm_adjoint(A, G)
    with pytest.raises(ValueError):
        mpps.expm_pade(np.zeros((3, 4)))
    with pytest.raises(ValueError):
        mpps.expm_pade(A, out=np.zeros((1, 4, 4)))
    with pytest.raises(ValueError):
        mpps.choose_s(30, 0.5, [1.0, 2.0], [1.0])
    # m < 1 is rejected by the C rule itself
    assert mpps.choose_s(0, 0.5, [1.0], [1.0]) == -1


def test_policy_struct_round_trip(mpps):
    """Every Policy field reaches the C struct in order (the struct has no padding surprises:
    its fields are read back through ctypes)."""
    p = mpps.Policy(mode=mpps.MIXED_PAPER, tol=1e-12, delta=7.0, s=5, formats=["fp64", "bf16"],
                    fp64_floor_steps=3, f64_slices=9, variable_s=True, adjoint_recompute=True)
    c = p._c()
    assert (c.mode, c.tol, c.delta, c.s, c.formats, c.fp64_floor_steps, c.f64_slices,
            c.variable_s, c.adjoint_recompute) == (mpps.MIXED_PAPER, 1e-12, 7.0, 5, 0b1001, 3, 9, 1, 1)
    d = mpps._Policy()
    mpps.lib().mpps_policy_default(d)
    assert (d.variable_s, d.adjoint_recompute, d.f64_slices, d.s) == (0, 0, 0, 0)


@pytest.mark.parametrize("mode", [oracle.MODE_FIXED, oracle.MODE_PAPER, oracle.MODE_NS])
def test_adjoint_planner_matches_oracle_rule(mpps, mode):
    """The reverse pass's rule (eq. (2.8) with u_i divided by m / min(1, ||X||_1)) agrees bit
    for bit with the oracle's statement."""
    rng = np.random.default_rng(70 + mode)
    for _ in range(300):
        m, n, norms, y = _rand_case(rng)
        x = float(10.0 ** rng.uniform(-3, 1))
        k = int(rng.choice([0, 8]))
        d = oracle.adjoint_divisor(m, x)
        ref = oracle.plan(m, n, norms, y, mode=mode, formats=0x1F, floor_steps=2, f64_slices=k,
                          divisor=d)
        got = mpps.plan_adjoint(m, n, norms, y, x, mpps.Policy(mode=mode, formats=0x1F,
                                                               fp64_floor_steps=2, f64_slices=k))
        assert got["nu"] == ref["nu"]
        for i in range(1, ref["r"] + 1):
            assert got["u"][i] == ref["u"][i], (m, i)
            want = ref["fmt"][i]
            assert got["fmt"][i] == (mpps.FORMAT_NAMES[want] if want is not None else None), (m, i)
        # tightening never asks for less precision than the forward rule
        fwd = oracle.plan(m, n, norms, y, mode=mode, formats=0x1F, floor_steps=2, f64_slices=k)
        for i in range(1, ref["r"] + 1):
            assert ref["u"][i] <= fwd["u"][i]


def test_adjoint_divisor_reading():
    assert oracle.adjoint_divisor(18, 9.0) == 18.0
    assert oracle.adjoint_divisor(18, 0.5) == 36.0
    assert oracle.adjoint_divisor(30, 0.0) == 30.0


# ---- mixed-precision powers: the leaf rule of the power tree ------------------------------
def _powers_case(rng):
    m = int(rng.integers(12, 60))
    s = oracle.ceil_sqrt(m)
    r = m // s
    coefs = [float(x) * (1.0 if rng.random() < 0.7 else -1.0)
             for x in 10.0 ** -np.cumsum(rng.uniform(0.0, 1.5, size=m + 1))]
    xp = [float(x) for x in 10.0 ** -np.cumsum(rng.uniform(0.0, 2.0, size=s))]
    nbp = [float(x) for x in 10.0 ** rng.uniform(-3, 1, size=r + 1)]
    if rng.random() < 0.1:
        xp[int(rng.integers(0, s))] = 0.0
    return m, s, coefs, xp, nbp


@pytest.mark.parametrize("k", [8, 9])
def test_plan_powers_matches_oracle_rule(mpps, k):
    """mpps_plan_powers agrees bit for bit with the oracle's statement of the leaf rule."""
    rng = np.random.default_rng(400 + k)
    pol = mpps.Policy(mode=mpps.MIXED_NS, f64_slices=k, mixed_powers=True)
    low = 0
    for _ in range(400):
        m, s, c, xp, nbp = _powers_case(rng)
        if s < 4:
            continue
        fmt, nb = mpps.plan_powers(m, s, c, xp, nbp, pol)
        ofmt, onb = oracle.plan_powers(m, s, c, xp, nbp, k)
        assert fmt == [mpps.FORMAT_NAMES[mpps.FMT_NONE if f is None else f] for f in ofmt], (m, s)
        assert list(nb) == onb
        low += sum(f != f"f64e{k}" for f in fmt[2:])
    assert low > 50          # the cases reach the cheaper rungs


def test_plan_powers_rejects(mpps):
    c, xp, nb = [1.0] * 17, [1.0] * 4, [1.0] * 5
    for pol in (mpps.Policy(f64_slices=8), mpps.Policy(mode=mpps.FIXED_FP64, f64_slices=8,
                                                       mixed_powers=True),
                mpps.Policy(f64_slices=0, mixed_powers=True)):
        with pytest.raises(mpps.MppsError) as e:
            mpps.plan_powers(16, 4, c, xp, nb, pol)
        assert e.value.status == 5
    with pytest.raises(mpps.MppsError):   # s = 3: no leaf
        mpps.plan_powers(9, 3, [1.0] * 10, [1.0] * 3, [1.0] * 4,
                         mpps.Policy(f64_slices=8, mixed_powers=True))


def test_plan_powers_bounds_hold_on_matrices():
    """Pins of the leaf rule against the matrices themselves (exact powers, plain norms):
    ||X^h|| ||X^(j-h)|| bounds ||X^j||, the norms handed to the block rule bound the true
    ones (below for B_0, above for i >= 1), and every cheaper leaf keeps its share of the
    budget: L ||X^h|| ||X^(j-h)|| S_j u_F64E(k_j) <= ||B_0||_low tol."""
    rng = np.random.default_rng(77)
    U = 2.0 ** -53
    for trial in range(40):
        n = 6
        m = int(rng.integers(16, 40))
        s = oracle.ceil_sqrt(m)
        r = m // s
        h = (s + 1) // 2
        X = rng.standard_normal((n, n))
        X *= float(10.0 ** rng.uniform(-1.5, 0)) / np.abs(X).sum(axis=0).max()
        c = [1.0 / math.factorial(i) for i in range(m + 1)] if trial % 2 else \
            [(-1) ** i * 0.5 ** i for i in range(m + 1)]
        P = [np.eye(n)]
        for _ in range(s):
            P.append(P[-1] @ X)
        n1 = lambda M: float(np.abs(M).sum(axis=0).max())
        leaves = set(range(h + 1, s))
        xp = [0.0 if j in leaves else n1(P[j]) for j in range(1, s + 1)]
        def block(i, with_leaves):
            B = np.zeros((n, n))
            for j in range(s):
                if s * i + j <= m and (with_leaves or j not in leaves):
                    B += c[s * i + j] * P[j]
            return B
        nbp = [n1(block(i, False)) for i in range(r + 1)]
        true = [n1(block(i, True)) for i in range(r + 1)]
        fmt, nb = oracle.plan_powers(m, s, c, xp, nbp, 8)
        for j in leaves:
            assert n1(P[j]) <= xp[h - 1] * xp[j - h - 1] * (1 + 1e-12)
        assert nb[0] <= true[0] * (1 + 1e-12)
        assert all(nb[i] >= true[i] * (1 - 1e-12) for i in range(1, r + 1))
        y = xp[s - 1]
        for j in leaves:
            k = fmt[j] - 16
            if k == 8:
                continue
            S = sum(abs(c[s * i + j]) * y ** i for i in range(r + 1) if s * i + j <= m)
            assert len(leaves) * xp[h - 1] * xp[j - h - 1] * S * 2.0 ** (2 - 7 * k) <= nb[0] * U * (1 + 1e-12)
