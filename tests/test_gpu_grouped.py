"""GPU checks of the grouped (uneven-batch) exp: the 4096-matrix configuration (n uniform in
[8, 256], ||A||_1 log-uniform in [0.1, 10], Taylor degree in {12, 18, 24}) with every matrix
checked against its own single-matrix evaluation and a sample against the double-double
oracle, and the whole grouped call captured in a CUDA graph and replayed."""
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


def test_grouped_4096_uneven_every_matrix(mpps):
    count = 4096
    mats, degs = inputs.uneven_batch(count, 8, 256, 0.1, 10.0, seed=3)
    dA = [dev(A) for A in mats]
    outs = mpps.expm_grouped(dA, degs, policy=mpps.NS_E)
    torch.cuda.synchronize()
    # every matrix: the grouped result and the matrix evaluated on its own both meet the
    # 50 n u 2^sigma bound, so they differ by at most twice it
    worst = 0.0
    for k in range(count):
        n = mats[k].shape[0]
        sg = oracle.sigma_for(mats[k])
        single = mpps.expm(dA[k], m=degs[k], policy=mpps.NS_E)
        d = (outs[k] - single).abs().sum(dim=0).max().item() / single.abs().sum(dim=0).max().item()
        bound = 2 * 50 * n * U * max(1, 2 ** sg)
        worst = max(worst, d / bound)
        assert d <= bound, (k, n, degs[k], sg, d)
    # a sample across the sizes against the oracle (double-double scaling and squaring)
    order = np.argsort([A.shape[0] for A in mats])
    sample = list(order[::400][:9]) + [int(order[-1])]
    for k in sample:
        A = mats[k]
        n, sg = A.shape[0], oracle.sigma_for(A)
        eh, el = oracle.expm_ss_dd(A, degs[k], sg)
        err = oracle.rel_err_1norm(outs[k].cpu().numpy(), eh, el)
        trunc = np.e / float(oracle.math.factorial(degs[k] + 1)) * 2 ** sg
        assert err <= 50 * n * U * max(1, 2 ** sg) + trunc, (k, n, degs[k], err)


def test_grouped_captured_in_a_cuda_graph(mpps):
    count = 60
    mats, degs = inputs.uneven_batch(count, 8, 140, 0.1, 10.0, seed=11)
    policy = dataclasses.replace(mpps.NS_E, max_squarings=5)   # ||A||_1 <= 10: sigma <= 4
    dA = [dev(A) for A in mats]
    outs = [torch.empty_like(a) for a in dA]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        mpps.expm_grouped(dA, degs, policy=policy, outs=outs)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        mpps.expm_grouped(dA, degs, policy=policy, outs=outs)
    new, _ = inputs.uneven_batch(count, 8, 140, 0.1, 10.0, seed=11)
    rng = np.random.default_rng(5)
    for k in range(count):   # new contents of the same shapes, other norms
        new[k] = new[k] * rng.uniform(0.2, 1.0)
        dA[k].copy_(dev(new[k]))
    g.replay()
    torch.cuda.synchronize()
    ref = mpps.expm_grouped([dev(A) for A in new], degs, policy=policy)
    for k in range(count):
        assert torch.equal(outs[k], ref[k]), k
    for k in (0, count // 2, count - 1):
        sg = oracle.sigma_for(new[k])
        eh, el = oracle.expm_ss_dd(new[k], degs[k], sg)
        n = new[k].shape[0]
        assert oracle.rel_err_1norm(outs[k].cpu().numpy(), eh, el) <= 50 * n * U * max(1, 2 ** sg) + \
            np.e / float(oracle.math.factorial(degs[k] + 1)) * 2 ** sg


def test_ps_eval_grouped_general_coefficients(mpps):
    """Uneven orders with three different coefficient sequences (Taylor exp, the Pade
    numerator, the Taylor cosine in B): each matrix against the oracle's PS in
    double-double, and its report against the single-matrix call's plan."""
    rng = np.random.default_rng(17)
    seqs = [(mpps.taylor_exp_coeffs(18), oracle.taylor_exp_rational(18)),
            (mpps.pade_exp_num_coeffs(13), oracle.pade_exp_num_rational(13)),
            (mpps.cos_taylor_coeffs(8), oracle.cos_taylor_rational(8))]
    ns = [5, 31, 33, 64, 70, 100, 129, 17, 48, 96, 1, 40]
    mats, coefs, rats = [], [], []
    for k, n in enumerate(ns):
        A = rng.standard_normal((n, n))
        A *= rng.uniform(0.2, 1.0) / np.abs(A).sum(axis=0).max()
        c, q = seqs[k % 3]
        mats.append(A); coefs.append(c); rats.append(q)
    outs, reps = mpps.ps_eval_grouped(coefs, [dev(A) for A in mats], policy=mpps.NS_E, report=True)
    for A, P, q, R in zip(mats, outs, rats, reps):
        n = A.shape[0]
        ph, pl, _ = oracle.ps_dd(q, A)
        assert oracle.rel_err_1norm(P.cpu().numpy(), ph, pl) <= 50 * n * U, n
        m = len(q) - 1
        assert (R["s"], R["r"]) == (oracle.ceil_sqrt(m), m // oracle.ceil_sqrt(m))


def test_shard_expm_local_two_ranks_in_sequence(mpps):
    """The multi-rank path on one GPU: rank 0 and rank 1 of a world of two evaluate their
    shards (shard.expm_local, no collective) one after the other; together they cover every
    matrix once and each result matches the oracle."""
    from paper_2312_17396_gb300 import shard
    mats, degs = inputs.uneven_batch(40, 8, 96, 0.1, 10.0, seed=23)
    dA = [dev(A) for A in mats]
    got = {}
    for rank in (0, 1):
        idx, outs = shard.expm_local(dA, degs, rank, 2, policy=mpps.NS_E)
        for i, E in zip(idx, outs):
            assert i not in got
            got[i] = E.cpu().numpy()
    assert sorted(got) == list(range(len(mats)))
    for i, A in enumerate(mats):
        n, sg = A.shape[0], oracle.sigma_for(A)
        eh, el = oracle.expm_ss_dd(A, degs[i], sg)
        trunc = np.e / float(oracle.math.factorial(degs[i] + 1)) * 2 ** sg
        assert oracle.rel_err_1norm(got[i], eh, el) <= 50 * n * U * max(1, 2 ** sg) + trunc, i
