"""GPU checks of the device-side precision plan (policy.device_plan): the rule of eq. (2.8)
runs on the GPU, every candidate format of a step is launched and all but the chosen one
return at once.  Its plans, scales and results must be the host planner's, bit for bit; with
blind squarings (policy.max_squarings) nothing is read back, so whole calls can be captured
in a CUDA graph and replayed."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2312_17396_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


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


def dp(pol, **kw):
    return dataclasses.replace(pol, device_plan=True, **kw)


def same_reports(ra, rb):
    for a, b in zip(ra, rb):
        for key in ("s", "r", "nu", "fmt", "u", "normB", "normY", "normX", "sigma", "gemms"):
            assert a[key] == b[key], (key, a[key], b[key])


@pytest.mark.parametrize("n,m", [(64, 30), (130, 12), (40, 24)])
@pytest.mark.parametrize("pol", ["paper", "ns", "paper_e", "ns_e", "fixed_e"])
def test_ps_eval_device_plan_is_the_host_plan(mpps, n, m, pol):
    policy = {"paper": mpps.PAPER, "ns": mpps.NS, "paper_e": mpps.PAPER_E, "ns_e": mpps.NS_E,
              "fixed_e": mpps.FIXED_E}[pol]
    A = inputs.gaussian_batch(3, n, seed=500 + n + m, norm1=[0.05, 0.4, 1.0])
    coef = mpps.taylor_exp_coeffs(m)
    P0, r0 = mpps.ps_eval(coef, dev(A), policy=policy, report=True)
    P1, r1 = mpps.ps_eval(coef, dev(A), policy=dp(policy), report=True)
    assert np.array_equal(host(P0), host(P1))
    same_reports(r0, r1)
    # without a report the call reads nothing back and gives the same bits
    P2 = mpps.ps_eval(coef, dev(A), policy=dp(policy))
    assert np.array_equal(host(P0), host(P2))


def test_ps_eval_device_plan_general_coefficients_fp8(mpps):
    """General signed coefficients and a loose target, so that FP8 and the emulated rungs are
    candidates: the device plan still equals the host plan."""
    n = 96
    A = inputs.gaussian_batch(2, n, seed=71, norm1=[0.3, 0.8])
    coef = np.array([1.0, -0.5, 0.25, 0.3, -0.2, 0.1, 0.05, -0.04, 0.01, 0.002, -0.001, 3e-4,
                     -1e-4, 2e-5, 1e-6, -3e-7, 1e-8])
    for tol in (2.0 ** -53, 2.0 ** -30):
        policy = dataclasses.replace(mpps.PAPER_E, tol=tol)
        P0, r0 = mpps.ps_eval(coef, dev(A), policy=policy, report=True)
        P1, r1 = mpps.ps_eval(coef, dev(A), policy=dp(policy), report=True)
        assert np.array_equal(host(P0), host(P1))
        same_reports(r0, r1)


@pytest.mark.parametrize("k", [0, 8])
@pytest.mark.parametrize("blind", [0, 7])
def test_expm_device_plan_is_the_host_plan(mpps, k, blind):
    n = 72
    A = inputs.gaussian_batch(4, n, seed=88, norm1=[0.3, 2.5, 9.0, 40.0])
    policy = mpps.Policy(mode=mpps.MIXED_NS, f64_slices=k)
    E0, r0 = mpps.expm(dev(A), policy=policy, report=True)
    E1, r1 = mpps.expm(dev(A), policy=dp(policy, max_squarings=blind), report=True)
    assert np.array_equal(host(E0), host(E1))
    same_reports(r0, r1)
    E2 = mpps.expm(dev(A), policy=dp(policy, max_squarings=blind))
    assert np.array_equal(host(E0), host(E2))


def test_blind_squarings_too_few(mpps):
    """A matrix that needs more squarings than max_squarings gets NaN, the others their
    result; a host-pointer call reports MPPS_ECHECK at once."""
    n = 32
    A = inputs.gaussian_batch(2, n, seed=9, norm1=[0.5, 100.0])     # sigma 0 and 7
    policy = dp(mpps.NS_E, max_squarings=3)
    with pytest.raises(mpps.MppsError) as e:
        mpps.expm(A, policy=policy)
    assert e.value.status == 6
    E = host(mpps.expm(dev(A), policy=policy))
    # the device error word is reported by the next call that checks it, and then cleared
    with pytest.raises(mpps.MppsError) as e:
        mpps.expm(A[:1], policy=mpps.NS_E)
    assert e.value.status == 6
    mpps.expm(A[:1], policy=mpps.NS_E)
    assert np.isnan(E[1]).all()
    eh, el = oracle.expm_ss_dd(A[0], 30, oracle.sigma_for(A[0]))
    assert oracle.rel_err_1norm(E[0], eh, el) <= 50 * n * U


def capture(fn):
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        fn()
    return g


@pytest.mark.parametrize("pol", ["ns_e", "paper"])
def test_ps_eval_captured_in_a_cuda_graph(mpps, pol):
    policy = dp({"ns_e": mpps.NS_E, "paper": mpps.PAPER}[pol])
    n, m = 128, 30
    coef = mpps.taylor_exp_coeffs(m)
    A = dev(inputs.gaussian_batch(2, n, seed=3, norm1=[0.2, 0.9]))
    out = torch.empty_like(A)
    g = capture(lambda: mpps.ps_eval(coef, A, policy=policy, out=out))
    for seed, norms in ((4, [0.9, 0.05]), (5, [0.5, 1.0])):
        Anew = inputs.gaussian_batch(2, n, seed=seed, norm1=norms)
        A.copy_(dev(Anew))
        g.replay()
        ref = mpps.ps_eval(coef, dev(Anew), policy=policy)
        assert np.array_equal(host(out), host(ref))
        ph, pl, _ = oracle.ps_dd(oracle.taylor_exp_rational(m), Anew[0])
        assert oracle.rel_err_1norm(host(out)[0], ph, pl) <= 50 * n * U


def test_expm_captured_in_a_cuda_graph(mpps):
    policy = dp(mpps.NS_E, max_squarings=6)
    n = 96
    A = dev(inputs.gaussian_batch(3, n, seed=21, norm1=[0.5, 4.0, 32.0]))
    out = torch.empty_like(A)
    g = capture(lambda: mpps.expm(A, policy=policy, out=out))
    Anew = inputs.gaussian_batch(3, n, seed=22, norm1=[20.0, 0.7, 3.0])
    A.copy_(dev(Anew))
    g.replay()
    ref = mpps.expm(dev(Anew), policy=mpps.NS_E)
    assert np.array_equal(host(out), host(ref))
