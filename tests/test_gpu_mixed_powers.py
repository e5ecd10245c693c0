"""GPU checks of the mixed-precision powers (policy.mixed_powers): the power tree whose leaves
X^(h+1)..X^(s-1) run in the slices mpps_plan_powers allows, against the double-double oracle
with the "mixed within 2x of fixed" criterion, the leaves' formats in the report, general
coefficients, and the cases where the option leaves the chain in place."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2312_17396_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
FLOOR = 4 * U   # "mixed within 2x of fixed" floor: a few ulps of ||P||


@pytest.fixture(scope="module")
def mpps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_17396_gb300 as m
    m.lib()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def c2(mpps, **kw):
    return dataclasses.replace(mpps.NS_E, formats=("fp64", "bf16x3", "tf32", "bf16"), **kw)


@pytest.mark.parametrize("norm", [0.5, 4.0, 32.0])
def test_expm_n1024_mixed_powers_sampled_columns(mpps, norm):
    """The headline configuration (n = 1024, m = 30, s = 6: chain X^2, X^3, Y = X^3 X^3,
    leaves X^4 = X^3 X, X^5 = X^3 X^2): within 2x of the fixed-FP64 error on sampled columns,
    and the leaves take fewer slices than the working precision."""
    n = 1024
    A = inputs.gaussian_matrix(n, seed=2, norm1=norm)
    sg = oracle.sigma_for(A)
    X = np.ldexp(A, -sg)
    cols = [0, 511, 1023]
    V = np.zeros((n, len(cols)))
    for t, j in enumerate(cols):
        V[j, t] = 1.0
    wh, wl = oracle.ps_apply_dd(oracle.taylor_exp_rational(30), X, V, reps=2 ** sg)
    ref_norm = np.abs(wh).sum(axis=0)
    errs = {}
    for name, pol in (("fixed", mpps.FIXED), ("c2", c2(mpps)), ("mixp", c2(mpps, mixed_powers=True))):
        E, rep = mpps.expm(dev(A), m=30, policy=pol, report=True)
        E = host(E)
        errs[name] = np.abs(E[:, cols] - wh - wl).sum(axis=0) / ref_norm
        if name == "mixp":
            pf = rep[0]["pow_fmt"]
            assert pf[:4] == ["none", "none", "f64e8", "f64e8"] and pf[6] == "f64e8", pf
            assert pf[4] != "f64e8" and pf[5] != "f64e8", pf   # both leaves cheaper
    assert np.all(errs["mixp"] <= 2 * errs["fixed"] + FLOOR), errs


@pytest.mark.parametrize("n", [64, 130])
def test_expm_mixed_powers_batch_vs_oracle(mpps, n):
    """A batch of three norms (sigma 0, 2, 5), m = 30: every matrix within 2x of fixed FP64
    against the full double-double result; the leaves run in the most precise format any
    matrix of the batch asks for."""
    A = inputs.gaussian_batch(3, n, seed=50 + n, norm1=[0.5, 4.0, 32.0])
    Ef = host(mpps.expm(dev(A), m=30, policy=mpps.FIXED))
    Em, rep = mpps.expm(dev(A), m=30, policy=c2(mpps, mixed_powers=True), report=True)
    Em = host(Em)
    for b in range(3):
        eh, el = oracle.expm_ss_dd(A[b], 30, oracle.sigma_for(A[b]))
        ef = oracle.rel_err_1norm(Ef[b], eh, el)
        em = oracle.rel_err_1norm(Em[b], eh, el)
        assert em <= 2 * ef + FLOOR, (b, em, ef)
        assert rep[b]["pow_fmt"] == rep[0]["pow_fmt"]


@pytest.mark.parametrize("m", [16, 24])
def test_ps_eval_mixed_powers_general_coefficients(mpps, m):
    """Algorithm 4.1 with general coefficients (the Pade numerator of degree 13 continued by
    decaying terms, signs alternating): mixed powers within 2x of the fixed error."""
    n = 96
    coef = np.array([(-1) ** j / (1.5 ** j * (j + 1)) for j in range(m + 1)])
    X = inputs.gaussian_matrix(n, seed=60 + m, norm1=1.5)
    ph, pl = oracle.ps_dd(coef, X)[:2]
    Pf = host(mpps.ps_eval(coef, dev(X), policy=mpps.FIXED))
    Pm, rep = mpps.ps_eval(coef, dev(X), policy=dataclasses.replace(mpps.NS_E, mixed_powers=True),
                           report=True)
    Pm = host(Pm)
    ef = oracle.rel_err_1norm(Pf, ph, pl)
    em = oracle.rel_err_1norm(Pm, ph, pl)
    assert em <= 2 * ef + FLOOR, (em, ef)
    s = rep[0]["s"]
    assert rep[0]["pow_fmt"][2] == "f64e8" and rep[0]["pow_fmt"][s] == "f64e8"


def test_mixed_powers_left_out_where_the_tree_is_not_formed(mpps):
    """With the device plan, a fixed mode, or s < 4 the option changes nothing: the same bits
    as without it, every power in the working precision."""
    n = 64
    A = inputs.gaussian_batch(2, n, seed=70, norm1=[0.5, 4.0])
    for pol in (dataclasses.replace(mpps.NS_E, device_plan=True), mpps.FIXED_E):
        E0 = host(mpps.expm(dev(A), m=30, policy=pol))
        E1, rep = mpps.expm(dev(A), m=30, policy=dataclasses.replace(pol, mixed_powers=True),
                            report=True)
        assert np.array_equal(host(E1), E0)
        assert all(f == "f64e8" for f in rep[0]["pow_fmt"][2:])
    E0 = host(mpps.expm(dev(A), m=8, policy=mpps.NS_E))           # s = 3
    E1 = host(mpps.expm(dev(A), m=8, policy=dataclasses.replace(mpps.NS_E, mixed_powers=True)))
    assert np.array_equal(E1, E0)


def test_expm_n1024_batched_step_vs_oracle(mpps):
    """The benchmarked step: the three matrices (||A||_1 = 0.5, 4, 32; sigma 0, 2, 5) in one
    batched call with mixed powers.  Each product has 384 tiles, so the F64E(8) products run
    whole tiles in the full waves and split the last wave (the leaves' F64E(6) and F64E(5)
    run whole tiles); the squarings slice only the matrices of their lists.  Sampled columns against the oracle,
    within 2x of the fixed-FP64 error, and the same result as three separate calls up to
    the bound."""
    n = 1024
    A = np.stack([inputs.gaussian_matrix(n, seed=2 + k, norm1=nrm)
                  for k, nrm in enumerate((0.5, 4.0, 32.0))])
    pol = c2(mpps, mixed_powers=True)
    Eb, rep = mpps.expm(dev(A), m=30, policy=pol, report=True)
    Eb = host(Eb)
    Ef = host(mpps.expm(dev(A), m=30, policy=mpps.FIXED))
    cols = [0, 511, 1023]
    for b in range(3):
        assert rep[b]["pow_fmt"][4] != "f64e8" and rep[b]["pow_fmt"][5] != "f64e8"
        sg = oracle.sigma_for(A[b])
        V = np.zeros((n, len(cols)))
        for t, j in enumerate(cols):
            V[j, t] = 1.0
        wh, wl = oracle.ps_apply_dd(oracle.taylor_exp_rational(30), np.ldexp(A[b], -sg), V,
                                    reps=2 ** sg)
        ref = np.abs(wh).sum(axis=0)
        em = np.abs(Eb[b][:, cols] - wh - wl).sum(axis=0) / ref
        ef = np.abs(Ef[b][:, cols] - wh - wl).sum(axis=0) / ref
        assert np.all(em <= 2 * ef + FLOOR), (b, em, ef)
        Es = host(mpps.expm(dev(A[b]), m=30, policy=pol))
        assert np.abs(Es - Eb[b]).sum(axis=0).max() <= 100 * n * U * 2 ** sg * np.abs(Es).sum(axis=0).max()
