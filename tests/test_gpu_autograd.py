"""GPU parity of differentiation: remap as an autograd Function whose backward is the inverse
remap, in-place chain sections whose backward is the adjoint kernel.  Gradients of the linear loss
sum_f c_f sum_i x_f must equal the oracle's chain gradient bit for bit (the oracle's gradient is
itself pinned to central finite differences of an fp64 forward in the CPU tests)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P
    return P


def _aos_tensor(wl, fields):
    return torch.from_numpy(np.stack(fields, axis=1).astype(np.float32)).cuda()


def _loss(lay, groups, c):
    total = None
    for g, t in zip(lay.groups, groups):
        w = torch.tensor([c[f] for f in g], dtype=torch.float32, device="cuda")
        term = (t * w).sum()
        total = term if total is None else total + term
    return total


def _grad_fields(wl, grad_aos):
    gh = grad_aos.cpu().numpy()
    return [np.ascontiguousarray(gh[:, f]) for f in range(wl.F)]


def _plans(P, wl, seed):
    rng = np.random.default_rng(seed)
    F = wl.F
    cands = [P.Layout.aos(F), P.Layout.soa(F)]
    for _ in range(3):
        order = [int(x) for x in rng.permutation(F)]
        cuts = sorted(set(int(x) for x in rng.integers(1, F, 5)))
        groups, prev = [], 0
        for c in cuts + [F]:
            groups.append(order[prev:c])
            prev = c
        cands.append(P.Layout(groups))
    plans = [[cands[0]] * len(wl.sections), [cands[1]] * len(wl.sections)]
    plans.append([cands[int(rng.integers(0, len(cands)))] for _ in wl.sections])      # many remaps
    plans.append([cands[(k // 5) % len(cands)] for k in range(len(wl.sections))])     # runs of 5
    return plans


@pytest.mark.parametrize("pi", range(4))
def test_gradient_equals_oracle(P, pi):
    from paper_1407_4859_gb300.autograd import DifferentiableProgram
    wl = synth.config5(n=(1 << 12) + 5, n_sections=64)
    fields = oracle.initial_fields(wl)
    st = [a.copy() for a in fields]
    want_g = oracle.chain_grad(wl.sections, st, wl.loss_weights)
    S = P.Schema(wl.dtypes)
    plan = _plans(P, wl, 7)[pi]
    x = _aos_tensor(wl, fields).requires_grad_(True)
    prog = DifferentiableProgram(S, wl.n, P.Layout.aos(wl.F), wl.sections, plan)
    lay, out = prog.forward([x])
    # forward state equals the oracle's final state
    got = [None] * wl.F
    for g, t in zip(lay.groups, out):
        th = t.detach().cpu().numpy()
        for j, f in enumerate(g):
            got[f] = np.ascontiguousarray(th[:, j])
    for f in range(wl.F):
        assert np.array_equal(got[f].view(np.uint32), st[f].view(np.uint32)), "state field %d" % f
    _loss(lay, out, wl.loss_weights).backward()
    gf = _grad_fields(wl, x.grad)
    for f in range(wl.F):
        assert np.array_equal(gf[f].view(np.uint32), want_g[f].view(np.uint32)), "grad field %d" % f
    # the inputs are left unchanged by the in-place sections
    assert np.array_equal(x.detach().cpu().numpy(), np.stack(fields, axis=1))


def test_remap_fn_backward_is_the_inverse_remap(P):
    from paper_1407_4859_gb300.autograd import RemapFn
    rng = np.random.default_rng(3)
    n, F = 3001, 9
    S = P.Schema([0] * F)
    src, dst = P.Layout([[0, 1, 2], [3], [4, 5, 6, 7, 8]]), P.Layout([[4, 5, 6, 7, 8], [2, 0], [1, 3]])
    xs = [torch.randn(n, len(g), device="cuda", requires_grad=True) for g in src.groups]
    moved_src = [xs[0], xs[1]]                                   # group [4..8] is shared
    outs = RemapFn.apply((S, n, src, dst, xs), *moved_src)
    gouts = [torch.randn_like(o) for o in outs]
    torch.autograd.backward(outs, gouts)
    # forward: fields moved; backward: gradient of field f lands where field f came from
    assert torch.equal(outs[0][:, 0], xs[0][:, 2].detach()) and torch.equal(outs[0][:, 1], xs[0][:, 0].detach())
    assert torch.equal(outs[1][:, 0], xs[0][:, 1].detach()) and torch.equal(outs[1][:, 1], xs[1][:, 0].detach())
    assert torch.equal(xs[0].grad[:, 2], gouts[0][:, 0]) and torch.equal(xs[0].grad[:, 0], gouts[0][:, 1])
    assert torch.equal(xs[0].grad[:, 1], gouts[1][:, 0]) and torch.equal(xs[1].grad[:, 0], gouts[1][:, 1])
    assert xs[2].grad is None


def test_full_size_gradient_sampled(P):
    """2^26 records x 24 fields (6.4 GB), 64 sections under a plan with several layout changes:
    forward state and gradient on 2048 sampled records equal the oracle's per-record values."""
    from paper_1407_4859_gb300.autograd import DifferentiableProgram
    wl = synth.config5()
    n = wl.n
    S = P.Schema(wl.dtypes)
    plan = _plans(P, wl, 7)[3]
    cols = [torch.from_numpy(wl.values(f)).cuda() for f in range(wl.F)]
    x = torch.stack(cols, dim=1).requires_grad_(True)
    del cols
    prog = DifferentiableProgram(S, n, P.Layout.aos(wl.F), wl.sections, plan)
    lay, out = prog.forward([x])
    rng = np.random.default_rng(5)
    idx = np.concatenate([[0, n - 1], rng.integers(0, n, 2048)])
    tsel = {}                      # read the forward state first: the backward restores it in place
    for g, t in zip(lay.groups, out):
        th = t.detach()[torch.from_numpy(idx).cuda()].cpu().numpy()
        for j, f in enumerate(g):
            tsel[f] = np.ascontiguousarray(th[:, j])
    _loss(lay, out, wl.loss_weights).backward()
    sf = [wl.values(f, idx=idx) for f in range(wl.F)]
    want_g = oracle.chain_grad(wl.sections, sf, wl.loss_weights)
    gsel = x.grad[torch.from_numpy(idx).cuda()].cpu().numpy()
    for f in range(wl.F):
        assert np.array_equal(np.ascontiguousarray(gsel[:, f]).view(np.uint32), want_g[f].view(np.uint32)), f
    for f in range(wl.F):
        assert np.array_equal(tsel[f].view(np.uint32), sf[f].view(np.uint32)), f


def test_differentiable_measure_prices_forward_and_backward(P):
    """ADHA_MEASURE_DIFFERENTIABLE: remap edges cost both directions (symmetric table), sections cost
    their forward launch with saves plus the adjoint kernel (more than the forward alone), and the plan
    PDL picks on that table trains bit for bit like the oracle."""
    from paper_1407_4859_gb300.autograd import DifferentiableProgram
    wl = synth.config5(n=(1 << 16) + 5, n_sections=12)
    n, F = wl.n, wl.F
    S, AOS = P.Schema(wl.dtypes), P.Layout.aos(F)
    fields = oracle.initial_fields(wl)
    x0 = _aos_tensor(wl, fields)
    secs = P.Sections(wl.sections)
    cand = P.adha_plan_sections(S, secs, P.PlanOpts([16, 32, 0], max_window=2, max_candidates=6))
    fwd = P.adha_measure(S, n, AOS, [x0], secs, cand)
    both = P.adha_measure(S, n, AOS, [x0], secs, cand, differentiable=True)
    L = len(cand)
    r = both.remap_ns
    assert all(r[a][b] == r[b][a] for a in range(L + 1) for b in range(L + 1))
    assert sum(map(sum, both.section_ns)) > sum(map(sum, fwd.section_ns))
    _, seq = P.adha_pdl_solve(both)
    plan = [cand.layouts[l] for l in seq]
    x = x0.detach().requires_grad_(True)
    lay, out = DifferentiableProgram(S, n, AOS, wl.sections, plan).forward([x])
    _loss(lay, out, wl.loss_weights).backward()
    torch.cuda.synchronize()
    want_g = oracle.chain_grad(wl.sections, [a.copy() for a in fields], wl.loss_weights)
    got = _grad_fields(wl, x.grad)
    for f in range(F):
        assert np.array_equal(got[f].view(np.uint32), want_g[f].view(np.uint32)), "gradient of field %d" % f
