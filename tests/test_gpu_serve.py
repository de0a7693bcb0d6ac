"""The continuous-batching server (rmc_server_*): every request's result is the same whether it runs alone or
in a mix of concurrently admitted requests (bit-identical: each request takes a route fixed by its own size
and precision, and neither route's arithmetic depends on other requests), admission respects the memory
budget, and every ticket completes exactly once."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    import paper_1505_07570_gb300 as rmc
    return rmc


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# (kind, m, n, k or s, p, q, sketch, prec): both routes, several sketch kinds and precisions
SPECS = [
    ("lsr", 3000, 64, 256, 0, 0, "countsketch", "fp32"),   # batched
    ("lsr", 5000, 300, 1200, 0, 0, "gaussian", "fp32"),    # n > 256: single-problem path
    ("lsr", 4000, 48, 192, 0, 0, "srht", "fp32"),          # not a count sketch: single-problem path
    ("lsr", 2000, 200, 800, 0, 0, "countsketch", "fp32"),  # batched
    ("rsvd", 3000, 100, 16, 8, 1, None, "fp32"),           # batched
    ("rsvd", 6000, 180, 32, 8, 1, None, "fp32"),           # l = 40: single-problem path
    ("rsvd", 4000, 120, 16, 8, 1, None, "tf32"),           # TF32 products: single-problem path
    ("rsvd", 800, 40, 8, 0, 0, None, "fp32"),              # batched, q = 0
    ("rsvd", 2500, 90, 12, 8, 1, None, "tf32x3"),          # 3xTF32: batched (FP32-level products)
]


def make(i, spec):
    kind, m, n, ks, p, q, sketch, prec = spec
    sp = dict(kind=kind, m=m, n=n, seed=500 + i)
    if kind == "rsvd":
        sp.update(k=ks, p=p, q=q)
    else:
        sp.update(s=ks)
    A, b = workloads.batch_problem_numpy(sp)
    return sp, dev(A), (dev(b) if b is not None else None), sketch or "countsketch", prec


def new_request(R, sp, A, b):
    if sp["kind"] == "rsvd":
        return R.rsvd_request(A, sp["k"], sp["p"], sp["q"], sp["seed"])
    return R.lsr_request(A, b, sp["s"], sp["seed"])


def direct(R, sp, A, b, sketch, prec):
    """The request through the entry point its route uses, alone."""
    if sp["kind"] == "lsr":
        if sketch == "countsketch" and sp["n"] <= 256 and sp["s"] <= 1024:
            r, x = R.lsr_request(A, b, sp["s"], sp["seed"])
            R.rmc_batch_run([r])
            return (x,)
        return (R.rmc_lsr_sketch(A, b, sp["s"], sketch, sp["seed"], prec=prec),)
    if prec in ("fp32", "tf32x3") and sp["k"] + sp["p"] <= 32 and sp["n"] <= 256:
        r, out = R.rsvd_request(A, sp["k"], sp["p"], sp["q"], sp["seed"])
        R.rmc_batch_run([r])
        return out
    return R.rmc_rsvd(A, sp["k"], sp["p"], sp["q"], sp["seed"], prec=prec)


@pytest.fixture(scope="module")
def problems(R):
    probs = [make(i, s) for i, s in enumerate(SPECS)]
    refs = [direct(R, *p) for p in probs]
    R.rmc_sync()
    return probs, refs


def outputs(o):
    return o if isinstance(o, tuple) else (o,)


def run_server(R, probs, waves, nstreams=4, budget=8 << 30):
    """Submit the problems in `waves` (lists of indices) with progress calls in between; returns outputs."""
    srv = R.Server(budget, nstreams=nstreams, max_batch=64)
    outs, tickets = {}, {}
    for wave in waves:
        for i in wave:
            sp, A, b, sketch, prec = probs[i]
            r, o = new_request(R, sp, A, b)
            outs[i] = outputs(o)
            tickets[srv.submit(r, sketch=sketch, prec=prec)] = i
        srv.progress()
    srv.drain()
    done = srv.poll()
    srv.close()
    assert sorted(t for t, _, _ in done) == sorted(tickets)
    assert all(st == R.RMC_OK for _, st, _ in done)
    assert all(lat >= 0 for _, _, lat in done)
    return outs


def test_serve_all_at_once_equals_alone(R, problems):
    probs, refs = problems
    outs = run_server(R, probs, [list(range(len(probs)))])
    for i, ref in enumerate(refs):
        for g, e in zip(outs[i], outputs(ref)):
            assert torch.equal(g, e), SPECS[i]


def test_serve_interleaved_equals_alone(R, problems):
    """Requests arriving while others are in flight (several waves, one stream and two streams)."""
    probs, refs = problems
    waves = [[0, 4], [1, 5, 7], [2, 8], [3, 6]]
    for nstreams in (1, 2):
        outs = run_server(R, probs, waves, nstreams=nstreams)
        for i, ref in enumerate(refs):
            for g, e in zip(outs[i], outputs(ref)):
                assert torch.equal(g, e), (nstreams, SPECS[i])


def test_serve_eight_lanes_repeated_mix(R, problems):
    """Eight lanes, each issuing its launches from its own host thread, on the mix repeated four times: every
    request completes without error and equals the request alone (kernels whose shared-memory cap depends on
    the problem are launched from several threads at once)."""
    probs, refs = problems
    waves = [list(range(len(probs)))] * 4
    srv_outs = []
    srv = R.Server(8 << 30, nstreams=8, max_batch=64)
    tickets = {}
    for w, wave in enumerate(waves):
        for i in wave:
            sp, A, b, sketch, prec = probs[i]
            r, o = new_request(R, sp, A, b)
            srv_outs.append((i, outputs(o)))
            tickets[srv.submit(r, sketch=sketch, prec=prec)] = len(srv_outs) - 1
        srv.progress()
    srv.drain()
    done = srv.poll()
    srv.close()
    assert sorted(t for t, _, _ in done) == sorted(tickets)
    assert all(st == R.RMC_OK for _, st, _ in done), [st for _, st, _ in done if st != R.RMC_OK]
    for i, outs in srv_outs:
        for g, e in zip(outs, outputs(refs[i])):
            assert torch.equal(g, e), SPECS[i]


def test_serve_budget_and_invalid(R, problems):
    probs, _ = problems
    srv = R.Server(1 << 20, nstreams=1, max_batch=8)   # 1 MB: too small for the n = 300 least squares
    sp, A, b, sketch, prec = probs[1]
    r, x = new_request(R, sp, A, b)
    with pytest.raises(R.RmcError) as e:
        srv.submit(r, sketch=sketch, prec=prec)
    assert e.value.status == R.RMC_ENOMEM
    sp, A, b, sketch, prec = probs[0]
    r, x = new_request(R, sp, A, b)
    r.s = 10  # s < n
    with pytest.raises(R.RmcError) as e:
        srv.submit(r, sketch=sketch, prec=prec)
    assert e.value.status == R.RMC_EINVAL
    srv.close()


def test_served_results_match_the_oracle(R, problems):
    """Each served result against the FP64 oracle on the same FP32 inputs: least squares x within 1e-4 relative,
    k-SVD singular values within 1e-4 (2e-3 for single-TF32 products) and ||A - U S V^T||_F within 1% of the
    oracle's."""
    from oracle import lsr, rsvd
    probs, _ = problems
    outs = run_server(R, probs, [list(range(len(probs)))], nstreams=2)
    for i, (sp, A, b, sketch, prec) in enumerate(probs):
        Ah = A.cpu().numpy()
        if sp["kind"] == "lsr":
            xo = lsr.lsr_sketch(Ah, b.cpu().numpy(), sp["s"], sketch, sp["seed"])
            x = outs[i][0].cpu().numpy()
            assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-4, SPECS[i]
        else:
            U, s, V = (t.cpu().numpy().astype(np.float64) for t in outs[i])
            Uo, so, Vo, _ = rsvd.rsvd(Ah, sp["k"], sp["p"], sp["q"], sp["seed"])
            np.testing.assert_allclose(s, so, rtol=2e-3 if prec == "tf32" else 1e-4, err_msg=str(SPECS[i]))
            A64 = Ah.astype(np.float64)
            err = np.linalg.norm(A64 - (U * s) @ V.T)
            erro = np.linalg.norm(A64 - (Uo * so) @ Vo.T)
            assert abs(err - erro) <= 0.01 * erro, SPECS[i]


# ------------------------------------------------------------------------ resident least-squares state
# With residency on, every least-squares request takes the resident route: S^T A and its factor are kept per
# (matrix, sketch) and a later request only sketches its own b and refines.  Its result must not depend on what
# is resident (first request, repeat, evicted, or no room at all), must match the oracle, and must follow a
# matrix that changed after rmc_server_release.
LSR_IDX = [i for i, sp in enumerate(SPECS) if sp[0] == "lsr"]


def run_resident(R, probs, order, cap, nstreams=2, rhs=None):
    """Least-squares requests `order` (problem indices; repeats reuse a problem's resident state) on a server
    with a resident cap of `cap` bytes; rhs[pos] replaces the problem's b at position pos.  Returns the x's."""
    srv = R.Server(8 << 30, nstreams=nstreams, max_batch=64)
    srv.resident(cap)
    outs, tickets = [], {}
    for pos, i in enumerate(order):
        sp, A, b, sketch, prec = probs[i]
        r, x = R.lsr_request(A, b if rhs is None else rhs[pos], sp["s"], sp["seed"])
        outs.append(x)
        tickets[srv.submit(r, sketch=sketch, prec=prec)] = pos
        if pos % 2:
            srv.progress()
    srv.drain()
    done = srv.poll()
    srv.close()
    assert sorted(t for t, _, _ in done) == sorted(tickets)
    assert all(st == R.RMC_OK for _, st, _ in done)
    return outs


def test_resident_results_do_not_depend_on_residency(R, problems):
    probs, _ = problems
    order = LSR_IDX * 3
    roomy = run_resident(R, probs, order, 1 << 30)
    one_entry = run_resident(R, probs, order, 2 << 20, nstreams=1)   # evictions between problems
    no_room = run_resident(R, probs, order, 1)                        # never resident, same route
    for pos in range(len(order)):
        first = order.index(order[pos])
        assert torch.equal(roomy[pos], roomy[first]), SPECS[order[pos]]
        assert torch.equal(one_entry[pos], roomy[pos]), SPECS[order[pos]]
        assert torch.equal(no_room[pos], roomy[pos]), SPECS[order[pos]]


def test_resident_results_match_the_oracle(R, problems):
    """x within 1e-4 of the FP64 oracle's sketch-and-solve on the same inputs, for each problem's own b and two
    fresh right-hand sides per problem (served against the resident sketch)."""
    from oracle import lsr
    probs, _ = problems
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    order, rhs = [], []
    for i in LSR_IDX:
        b = probs[i][2]
        for j in range(3):
            order.append(i)
            rhs.append(b if j == 0 else torch.randn(b.shape[0], generator=gen, device="cuda"))
    outs = run_resident(R, probs, order, 1 << 30, rhs=rhs)
    for pos, i in enumerate(order):
        sp, A, _, sketch, _ = probs[i]
        xo = lsr.lsr_sketch(A.cpu().numpy(), rhs[pos].cpu().numpy(), sp["s"], sketch, sp["seed"])
        x = outs[pos].cpu().numpy()
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-4, SPECS[i]


def test_resident_state_released_with_its_matrix(R, problems):
    """After rmc_server_release(A), a changed A is sketched and factored again: doubling A halves x."""
    probs, _ = problems
    sp, A, b, sketch, prec = probs[LSR_IDX[0]]
    A2 = A.clone()
    srv = R.Server(8 << 30, nstreams=1, max_batch=8)
    srv.resident(1 << 30)
    r, x1 = R.lsr_request(A2, b, sp["s"], sp["seed"])
    srv.submit(r, sketch=sketch, prec=prec)
    srv.drain()
    A2.mul_(2.0)
    srv.release(A2)
    r, x2 = R.lsr_request(A2, b, sp["s"], sp["seed"])
    srv.submit(r, sketch=sketch, prec=prec)
    srv.drain()
    assert all(st == R.RMC_OK for _, st, _ in srv.poll())
    srv.close()
    torch.testing.assert_close(x2 * 2, x1, rtol=1e-5, atol=1e-7)
