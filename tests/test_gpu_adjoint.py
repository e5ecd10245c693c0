"""GPU checks of the reverse pass through its tape (ps_eval_forward_tape /
ps_eval_adjoint_tape) and of the mixed-precision reverse Horner products.

Tolerances: gradients within 100 n 2^-53 of the double-double oracle (the adjoint's bound
used throughout), and a mixed-precision gradient within 2x of the fixed-FP64 gradient's
error up to 4 ulps of ||grad|| (the forward rule's acceptance bar, applied to the reverse
pass)."""
import numpy as np
import pytest

import oracle
from paper_2312_17396_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
FLOOR = 4 * U
HDR_INTS = 8 + 2 * 65          # TapeHeader: 8 ints, fmt[65], fmt_adj[65]


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


def header(tape):
    """The formats of both passes, read from the tape's header (its last bytes)."""
    torch.cuda.synchronize()
    raw = tape[-4 * HDR_INTS:].cpu().numpy().view(np.int32)
    r = int(raw[5])
    return list(raw[8 + 1:8 + 1 + r]), list(raw[8 + 65 + 1:8 + 65 + 1 + r])


def rank(f):
    """Precision order of the formats: FP8 < BF16 < TF32 < BF16X3 < F64E(k) < FP64."""
    f = int(f)
    if f == 0:
        return 1000
    if f > 16:
        return 100 + (f - 16)
    return {1: 4, 2: 3, 3: 2, 4: 1}[f]


def case(n, m, norm, seed):
    A = inputs.gaussian_matrix(n, seed=seed, norm1=norm)
    G = np.random.default_rng(seed + 1).standard_normal((n, n))
    gh, gl = oracle.adjoint_dd(oracle.taylor_exp_rational(m), A, G)
    return A, G, gh, gl


@pytest.mark.parametrize("n,m,norm", [(33, 18, 0.3), (64, 30, 0.7), (130, 18, 1.0), (64, 13, 0.05)])
def test_adjoint_mixed_within_2x_of_fixed(mpps, n, m, norm):
    A, G, gh, gl = case(n, m, norm, 4000 + n + m)
    coef = mpps.taylor_exp_coeffs(m)
    rel = lambda g: oracle.norm1(g - gh - gl) / oracle.norm1(gh)
    ef = rel(host(mpps.ps_eval_adjoint(coef, dev(A), dev(G), policy=mpps.FIXED)))
    assert ef <= 100 * n * U
    lowered = 0
    for pol in (mpps.PAPER, mpps.NS, mpps.PAPER_E, mpps.NS_E):
        e = rel(host(mpps.ps_eval_adjoint(coef, dev(A), dev(G), policy=pol)))
        assert e <= 100 * n * U, (pol.mode, pol.f64_slices, e)
        assert e <= 2 * ef + FLOOR, (pol.mode, pol.f64_slices, e, ef)
        _, tape = mpps.ps_eval_forward_tape(coef, dev(A), policy=pol)
        fmts, fadj = header(tape)
        wp = 0 if pol.f64_slices == 0 else mpps.FMT_F64E(pol.f64_slices)
        lowered += sum(1 for f in fadj if f != wp)
        # the reverse rule never runs a step below the forward step's precision
        for f, a in zip(fmts, fadj):
            if f >= 0:
                assert rank(a) >= rank(f), (fmts, fadj)
    if norm <= 0.3:
        assert lowered > 0     # the reverse pass does drop precision on small-norm inputs


@pytest.mark.parametrize("pol", ["fixed", "ns", "ns_e", "paper_e"])
def test_tape_forward_equals_ps_eval(mpps, pol):
    policy = {"fixed": mpps.FIXED, "ns": mpps.NS, "ns_e": mpps.NS_E, "paper_e": mpps.PAPER_E}[pol]
    A = inputs.gaussian_batch(3, 96, seed=77, norm1=[0.2, 0.9, 2.5])
    coef = mpps.taylor_exp_coeffs(24)
    P = host(mpps.ps_eval(coef, dev(A), policy=policy))
    Pt, _ = mpps.ps_eval_forward_tape(coef, dev(A), policy=policy)
    assert np.array_equal(P, host(Pt))


def test_autograd_backward_reuses_the_forward(mpps):
    """The backward pass of PolyFn runs only the reverse products: 2 per reverse Horner step
    and 2 per power, none of the forward's (s - 1 + r) products again."""
    n, m, batch = 64, 18, 2          # s = 5, r = 3, s does not divide m
    rng = np.random.default_rng(9)
    A = torch.tensor(rng.standard_normal((batch, n, n)) / np.sqrt(n), device="cuda:0",
                     dtype=torch.float64, requires_grad=True)
    coef = mpps.taylor_exp_coeffs(m)
    P = mpps.poly(A, coef, mpps.FIXED_E)
    G = torch.randn(P.shape, generator=torch.Generator(device="cuda:0").manual_seed(3),
                    device="cuda:0", dtype=P.dtype)
    torch.cuda.synchronize()
    mpps.profile_enable(True)
    mpps.profile_reset()
    P.backward(G)
    torch.cuda.synchronize()
    products = sum(mpps.profile_read(c)[0] for c in (mpps.PROF_GEMM_F64, mpps.PROF_GEMM_F64E,
                                                      mpps.PROF_GEMM_TC))
    mpps.profile_enable(False)
    s, r = 5, 3
    assert products == 2 * r + 2 * (s - 1)
    for b in range(batch):
        gh, gl = oracle.adjoint_dd(oracle.taylor_exp_rational(m), A[b].detach().cpu().numpy(),
                                   G[b].cpu().numpy())
        assert oracle.norm1(A.grad[b].cpu().numpy() - gh - gl) / oracle.norm1(gh) <= 100 * n * U


def test_adjoint_f32_entry_is_the_f64_path_rounded(mpps):
    """FP32 storage: the entry widens exactly and evaluates in FP64, so its gradient is the
    FP64 gradient of the widened inputs rounded to FP32, bit for bit."""
    n, m, batch = 128, 18, 3
    rng = np.random.default_rng(12)
    A32 = torch.tensor(rng.standard_normal((batch, n, n)) / np.sqrt(n), dtype=torch.float32,
                       device="cuda:0")
    G32 = torch.tensor(rng.standard_normal((batch, n, n)), dtype=torch.float32, device="cuda:0")
    coef = mpps.taylor_exp_coeffs(m)
    for pol in (mpps.FIXED_E, mpps.NS_E):
        g32 = mpps.ps_eval_adjoint_f32(coef, A32, G32, policy=pol)
        g64 = mpps.ps_eval_adjoint(coef, A32.double(), G32.double(), policy=pol)
        assert torch.equal(g32, g64.float())
        # and through the tape entry points with FP32 storage
        P32, tape = mpps.ps_eval_forward_tape(coef, A32, policy=pol)
        P64 = mpps.ps_eval(coef, A32.double(), policy=pol)
        assert torch.equal(P32, P64.float())
        assert torch.equal(mpps.ps_eval_adjoint_tape(coef, tape, G32, policy=pol), g32)


def test_tape_of_another_call_is_rejected(mpps):
    A = dev(inputs.gaussian_batch(2, 16, seed=3, norm1=[0.5, 0.5]))
    G = torch.ones_like(A)
    _, tape = mpps.ps_eval_forward_tape(mpps.taylor_exp_coeffs(12), A, policy=mpps.FIXED)
    with pytest.raises(mpps.MppsError) as e:
        mpps.ps_eval_adjoint_tape(mpps.taylor_exp_coeffs(16), tape, G, policy=mpps.FIXED)
    assert e.value.status == 1
    with pytest.raises(mpps.MppsError):
        mpps.ps_eval_adjoint_tape(mpps.taylor_exp_coeffs(12), tape, G[:1].contiguous(),
                                  policy=mpps.FIXED)


@pytest.mark.parametrize("k", [0, 8])
def test_expm_adjoint_mixed_within_2x_of_fixed(mpps, k):
    """Through scaling and squaring: the polynomial's two passes under the mixed rule, the
    squarings in the working precision."""
    n, m = 48, 30
    A = inputs.gaussian_batch(3, n, seed=61, norm1=[0.4, 3.0, 11.0])
    G = np.random.default_rng(62).standard_normal((3, n, n))
    gf = host(mpps.expm_adjoint(dev(A), dev(G), m=m, policy=mpps.Policy(mode=mpps.FIXED_FP64,
                                                                         f64_slices=k)))
    gm = host(mpps.expm_adjoint(dev(A), dev(G), m=m, policy=mpps.Policy(mode=mpps.MIXED_PAPER,
                                                                         f64_slices=k)))
    for b in range(3):
        sg = oracle.sigma_for(A[b])
        gh, gl = oracle.expm_ss_adjoint_dd(A[b], G[b], m, sg)
        ef = oracle.norm1(gf[b] - gh - gl) / oracle.norm1(gh)
        em = oracle.norm1(gm[b] - gh - gl) / oracle.norm1(gh)
        assert em <= 100 * n * U * max(1, 2 ** sg) and em <= 2 * ef + FLOOR, (b, sg, em, ef)
