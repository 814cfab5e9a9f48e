"""Dirichlet elimination, batched Jacobi-CG and the request loop vs the CPU oracle (GB300 machine).

* Dirichlet: the CUDA kernel and the oracle rewrite the same assembled system; the matrix must
  match bitwise (only zeros and ones are written) and b within 1e-14 of the lift's scale.
* CG: the oracle's CG on the same system; both stop at ||r|| <= rtol ||b|| (rtol 1e-8), so
  ||x_gpu - x_oracle||_2 <= 2 rtol ||b|| / lambda_min(A) (the error bound of a residual), the
  iteration counts agree within 2 and the true residual of the GPU iterate is <= 2 rtol ||b||.
* Batching: a system's iterates are bitwise the same alone and beside others, with or without
  the CUDA graph, whatever tick lengths are used.
* Serving: every request's solution is bitwise the same in a mixed run and in the plain
  one-at-a-time run, satisfies the residual bound against the oracle's system, and the server
  never holds more device memory than its budget.
"""
import numpy as np
import pytest

import oracle as O
from paper_1501_01809_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_01809_gb300 import build
    build.build()
    return torch


class System:
    """A Poisson system assembled on the GPU (pull, FP64) with its device objects."""

    def __init__(self, ctx, n, p, k=1, m=2, jitter=0.0, seed=0, precision=0):
        import torch
        from paper_1501_01809_gb300 import fe
        self.fe, self.torch = fe, torch
        self.mesh = mg.unit_square_mesh(n, jitter, seed)
        self.cmap, self.nn = mg.cell_node_map(self.mesh, p)
        self.p = p
        self.f, self.u = mg.manufactured_sine(self.mesh, p, k, m)
        self.bc = mg.boundary_nodes(self.mesh, p)
        dev = torch.device("cuda", 0)
        self.t = {k_: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k_, v in
                  dict(map=self.cmap, cv=self.mesh.cell_vertex, xy=self.mesh.coords, f=self.f, bc=self.bc).items()}
        self.t["b"] = torch.zeros(self.nn, dtype=torch.float64, device=dev)
        self.t["x"] = torch.zeros(self.nn, dtype=torch.float64, device=dev)
        self.cells, self.nodes = fe.set_create(ctx, self.mesh.ncell), fe.set_create(ctx, self.nn)
        self.verts = fe.set_create(ctx, self.mesh.nvert)
        self.M = fe.map_create(ctx, self.cells, self.nodes, self.t["map"])
        self.CM = fe.map_create(ctx, self.cells, self.verts, self.t["cv"])
        self.XY = fe.dat_create(ctx, self.verts, self.t["xy"])
        self.F = fe.dat_create(ctx, self.nodes, self.t["f"])
        self.B = fe.dat_create(ctx, self.nodes, self.t["b"])
        self.X = fe.dat_create(ctx, self.nodes, self.t["x"])
        self.sp = fe.sparsity_build(ctx, self.M, self.M)
        self.A = fe.mat_create(ctx, self.sp)
        kl = fe.kernel_create(ctx, fe.FORM_LAPLACE, 2, p, precision=precision, strategy=fe.STRATEGY_PULL)
        ks = fe.kernel_create(ctx, fe.FORM_SOURCE, 2, p, coeff_degree=p, precision=precision,
                              strategy=fe.STRATEGY_PULL)
        fe.assemble_mat(ctx, kl, self.cells, self.A, self.XY, self.CM, zero_first=True)
        fe.assemble_vec(ctx, ks, self.cells, self.B, self.M, self.XY, self.CM, [(self.F, self.M)], zero_first=True,
                        sp=self.sp)
        fe.sync(ctx)
        _, _, _, rp, ci = fe.sparsity_csr(self.sp)
        self.rp, self.ci = rp.cpu().numpy(), ci.cpu().numpy()

    def host(self):
        return self.fe.mat_values(self.A).cpu().numpy(), self.t["b"].cpu().numpy()


def _ctx():
    from paper_1501_01809_gb300 import fe
    return fe.ctx_create(0)


def test_dirichlet_matches_oracle(gpu):
    from paper_1501_01809_gb300 import fe
    ctx = _ctx()
    for n, p in [(9, 2), (33, 1), (4, 2)]:
        s = System(ctx, n, p, jitter=0.2, seed=n)
        v0, b0 = s.host()
        g = np.random.default_rng(n).uniform(-1, 1, s.nn)
        for gg in (None, g):
            s2 = System(ctx, n, p, jitter=0.2, seed=n)
            tg = None if gg is None else gpu.from_numpy(gg).cuda()
            fe.dirichlet_apply(ctx, s2.A, s2.B, s2.t["bc"], tg)
            fe.sync(ctx)
            vg, bg = s2.host()
            vo, bo = O.dirichlet_apply(s.rp, s.ci, v0, b0, s.bc, gg)
            np.testing.assert_array_equal(vg, vo)
            absA = np.abs(v0)
            lift = np.zeros(s.nn) if gg is None else np.array(
                [np.sum(absA[s.rp[i]:s.rp[i + 1]] * np.abs(gg[s.ci[s.rp[i]:s.rp[i + 1]]])) for i in range(s.nn)])
            scale = np.abs(b0) + lift + 1e-300
            assert np.all(np.abs(bg - bo) <= 1e-14 * scale), np.max(np.abs(bg - bo) / scale)


def _run_engine(cg, slots, tick=8, use_graph=True, maxticks=100000):
    from paper_1501_01809_gb300 import fe
    for _ in range(maxticks):
        fe.cg_iterate(cg, tick, use_graph)
        st, it, rn, bn = fe.cg_poll(cg, max(slots) + 1)
        if all(st[s] != fe.CG_RUNNING for s in slots):
            return st, it, rn, bn
    raise AssertionError("CG did not finish")


@pytest.mark.parametrize("n,p", [(12, 1), (31, 1), (9, 2), (24, 2), (90, 2)])
def test_cg_matches_oracle(gpu, n, p):
    from paper_1501_01809_gb300 import fe
    sp = pytest.importorskip("scipy.sparse")
    if n > 40:
        pytest.importorskip("scipy.sparse.linalg")
    ctx = _ctx()
    s = System(ctx, n, p, k=2, m=3, jitter=0.15, seed=1)
    fe.dirichlet_apply(ctx, s.A, s.B, s.t["bc"])
    fe.sync(ctx)
    v, b = s.host()
    cg = fe.cg_create(ctx, 4)
    slot = fe.cg_add(cg, s.A, s.B, s.X, rtol=1e-8)
    st, it, rn, bn = _run_engine(cg, [slot])
    x = s.t["x"].cpu().numpy()
    xo, ito, rno, bno = O.cg_jacobi(s.rp, s.ci, v, b, rtol=1e-8)
    assert st[slot] == fe.CG_CONVERGED and ito > 0
    assert abs(int(it[slot]) - ito) <= 2, (it[slot], ito)
    A = sp.csr_matrix((v, s.ci, s.rp), shape=(s.nn, s.nn))
    bnorm = np.linalg.norm(b)
    assert abs(bn[slot] - bnorm) <= 1e-12 * bnorm and rn[slot] <= 1e-8 * bn[slot]
    assert np.linalg.norm(b - A @ x) <= 2e-8 * bnorm
    if n > 40:  # smallest eigenvalue by shift-invert Lanczos (the dense matrix would be 33k x 33k)
        from scipy.sparse.linalg import eigsh
        lam_min = eigsh(A.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    else:
        lam_min = np.linalg.eigvalsh(A.toarray())[0]
    assert np.linalg.norm(x - xo) <= 2 * 2e-8 * bnorm / lam_min, (np.linalg.norm(x - xo), bnorm / lam_min)


def test_cg_alone_vs_mix_bitwise(gpu):
    from paper_1501_01809_gb300 import fe
    ctx = _ctx()
    specs = [(40, 2, 1, 1), (10, 1, 2, 2), (25, 2, 3, 1), (60, 1, 1, 4), (7, 2, 4, 4)]

    def solve(which, tick, use_graph, cap=8, order=None):
        cg = fe.cg_create(ctx, cap)
        systems, slots = [], []
        for i in (order or which):
            s = System(ctx, *specs[i][:2], k=specs[i][2], m=specs[i][3], jitter=0.1, seed=i)
            fe.dirichlet_apply(ctx, s.A, s.B, s.t["bc"])
            slots.append(fe.cg_add(cg, s.A, s.B, s.X, rtol=1e-10))
            systems.append((i, s))
        st, it, rn, bn = _run_engine(cg, slots, tick, use_graph)
        return {i: (s.t["x"].cpu().numpy(), int(it[sl])) for (i, s), sl in zip(systems, slots)}

    alone = {i: solve([i], 16, True)[i] for i in range(len(specs))}
    mixed = solve(list(range(len(specs))), 5, True, order=[3, 1, 4, 0, 2])
    direct = solve(list(range(len(specs))), 7, False)
    for i in range(len(specs)):
        for other, what in ((mixed, "mixed"), (direct, "direct launches")):
            assert other[i][1] == alone[i][1], (i, what)
            np.testing.assert_array_equal(other[i][0], alone[i][0], err_msg=f"system {i} {what}")


def test_cg_status_codes(gpu):
    from paper_1501_01809_gb300 import fe
    ctx = _ctx()
    s = System(ctx, 8, 1)
    fe.dirichlet_apply(ctx, s.A, s.B, s.t["bc"])
    cg = fe.cg_create(ctx, 4)
    # maxit 3: stops with FE_CG_MAXIT after exactly 3 iterations
    a = fe.cg_add(cg, s.A, s.B, s.X, rtol=1e-12, maxit=3)
    # zero right-hand side: converged before the first iteration
    tz = gpu.zeros(s.nn, dtype=gpu.float64, device="cuda")
    tx = gpu.zeros(s.nn, dtype=gpu.float64, device="cuda")
    Z, XZ = fe.dat_create(ctx, s.nodes, tz), fe.dat_create(ctx, s.nodes, tx)
    bz = fe.cg_add(cg, s.A, Z, XZ)
    st, it, rn, bn = _run_engine(cg, [a, bz], tick=2)
    assert st[a] == fe.CG_MAXIT and it[a] == 3
    assert st[bz] == fe.CG_CONVERGED and it[bz] == 0 and not tx.any()
    # a negated matrix is not SPD: reported as breakdown at set-up
    s2 = System(ctx, 8, 1)
    fe.dirichlet_apply(ctx, s2.A, s2.B, s2.t["bc"])
    fe.mat_values(s2.A).neg_()
    c2 = fe.cg_add(cg, s2.A, s2.B, s2.X)
    st, it, rn, bn = fe.cg_poll(cg, 4)
    assert st[c2] == fe.CG_BREAKDOWN
    fe.cg_remove(cg, a)
    st, it, rn, bn = fe.cg_poll(cg, 4)
    assert st[a] == -1


def _requests(specs):
    out = []
    for (t, n, p, k, m) in specs:
        mesh = mg.unit_square_mesh(n)
        cmap, nn = mg.cell_node_map(mesh, p)
        f, u = mg.manufactured_sine(mesh, p, k, m)
        out.append(dict(t=t, n=n, p=p, mesh=mesh, cmap=cmap, nn=nn, f=f, u=u, bc=mg.boundary_nodes(mesh, p)))
    return out


def _serve(reqs, budget, max_active, tick=8, keys=None, precision=0):
    from paper_1501_01809_gb300 import fe
    ctx = _ctx()
    srv = fe.server_create(ctx, budget, max_active=max_active, iters_per_tick=tick, rtol=1e-8, precision=precision)
    xs, ids = [], []
    for i, r in enumerate(reqs):
        x = np.full(r["nn"], np.nan)
        ids.append(fe.server_submit(srv, r["p"], r["cmap"], r["mesh"].cell_vertex, r["mesh"].coords, r["f"], r["bc"],
                                    x, r["t"], mesh_key=keys[i] if keys else 0))
        xs.append(x)
    fe.server_run(srv)
    return [fe.server_result(srv, i) for i in ids], xs, fe.server_stats(srv)


def test_server_mix_equals_alone_and_oracle(gpu):
    from paper_1501_01809_gb300 import fe
    sp = pytest.importorskip("scipy.sparse")
    specs = [(0.0, 24, 2, 1, 2), (0.0, 10, 1, 3, 1), (0.001, 50, 1, 2, 2), (0.002, 17, 2, 4, 3),
             (0.002, 8, 1, 1, 1), (0.004, 33, 2, 2, 4), (0.005, 70, 1, 1, 3), (0.006, 12, 2, 3, 3)]
    reqs = _requests(specs)
    res_mix, x_mix, stats = _serve(reqs, 1 << 34, 16)
    res_one, x_one, _ = _serve(reqs, 1 << 34, 1)
    assert stats["converged"] == len(reqs) and stats["estimate_misses"] == 0
    for i, r in enumerate(reqs):
        assert res_mix[i]["status"] == fe.SOLVE_CONVERGED and res_one[i]["status"] == fe.SOLVE_CONVERGED
        assert res_mix[i]["iters"] == res_one[i]["iters"]
        np.testing.assert_array_equal(x_mix[i], x_one[i], err_msg=f"request {i}: mixed vs alone")
        # residual of the served solution against the oracle's own assembled, eliminated system
        rp, ci = O.sparsity(r["cmap"], r["cmap"], r["nn"], r["nn"])
        v, _ = O.assemble_mat(2, r["p"], O.LAPLACE, r["cmap"], r["mesh"].coords, r["mesh"].cell_vertex, rp, ci)
        b, _ = O.assemble_vec(2, r["p"], r["p"], r["cmap"], r["nn"], r["mesh"].coords, r["mesh"].cell_vertex, r["f"],
                              r["cmap"])
        v, b = O.dirichlet_apply(rp, ci, v, b, r["bc"])
        A = sp.csr_matrix((v, ci, rp), shape=(r["nn"], r["nn"]))
        assert np.linalg.norm(b - A @ x_mix[i]) <= 1.5e-8 * np.linalg.norm(b), i
        # and it approximates the manufactured solution (discretisation error, not a parity bound)
        assert np.abs(x_mix[i] - r["u"]).max() < 0.1, i
        assert res_mix[i]["finished_s"] >= res_mix[i]["admitted_s"] >= specs[i][0]


@pytest.mark.parametrize("precision", [0, 1])
def test_server_round_equals_per_request_launches(gpu, precision):
    """Requests admitted together form one round: one element launch and one row launch assemble
    all of their systems, the boundary elimination fused into the row write-out.  Each system is
    bitwise the one the per-request calls give (pull assembly of the Mat and of the right-hand
    side, then the elimination kernel): its served solution and iteration count equal those of
    the same system built through the public calls and solved by the same CG, alone.  Element
    tensors in FP64 (precision 0) and in double-float (1)."""
    from paper_1501_01809_gb300 import fe
    specs = [(0.0, 24, 2, 1, 2), (0.0, 10, 1, 3, 1), (0.0, 50, 1, 2, 2), (0.0, 17, 2, 4, 3), (0.0, 2, 1, 1, 1),
             (0.0, 33, 2, 2, 4), (0.0, 3, 2, 1, 1)]
    reqs = _requests(specs)
    res, xs, stats = _serve(reqs, 1 << 34, 16, precision=precision)
    assert stats["converged"] == len(reqs) and stats["sparsity_builds"] == len(reqs)
    ctx = _ctx()
    for i, (_, n, p, k, m) in enumerate(specs):
        s = System(ctx, n, p, k=k, m=m, precision=precision)
        fe.dirichlet_apply(ctx, s.A, s.B, s.t["bc"])
        cg = fe.cg_create(ctx, 16)
        slot = fe.cg_add(cg, s.A, s.B, s.X, rtol=1e-8)
        st, it, _, _ = _run_engine(cg, [slot])
        assert st[slot] == fe.CG_CONVERGED and res[i]["iters"] == int(it[slot]), (i, res[i]["iters"], it[slot])
        np.testing.assert_array_equal(xs[i], s.t["x"].cpu().numpy(), err_msg=f"request {i}")


def test_server_request_out_of_range_fails_its_round(gpu):
    """A request whose cell-vertex map points past its vertices fails the round at the range
    check, before any kernel reads through that map: server_run reports FE_ERANGE naming the
    request, and the context serves the next server's requests as before."""
    from paper_1501_01809_gb300 import fe
    specs = [(0.0, 12, 2, 1, 1), (0.0, 9, 1, 2, 1), (0.0, 12, 1, 1, 2)]
    reqs = _requests(specs)
    bad = dict(reqs[1])
    bad["mesh"] = mg.unit_square_mesh(9)
    bad["mesh"].cell_vertex[5, 1] = bad["mesh"].nvert  # one past the last vertex
    with pytest.raises(fe.FeError) as ei:
        _serve([reqs[0], bad, reqs[2]], 1 << 34, 8, keys=[0, 3, 0])
    assert ei.value.code == fe.FE_ERANGE and "request 1" in str(ei.value), str(ei.value)
    res, xs, stats = _serve(reqs, 1 << 34, 8)
    assert stats["converged"] == len(reqs)
    ref, xr, _ = _serve(reqs, 1 << 34, 1)
    for a, b in zip(xs, xr):
        np.testing.assert_array_equal(a, b)


def test_server_budget_binds_and_refuses(gpu):
    from paper_1501_01809_gb300 import fe
    specs = [(0.0, 40, 2, 1, 1), (0.0, 40, 2, 2, 1), (0.0, 40, 2, 1, 2), (0.0, 20, 1, 1, 1), (0.0, 300, 2, 1, 1)]
    reqs = _requests(specs)
    # room for one 40x40 P2 request at a time (its worst case plus half of what it holds once
    # built); the 300x300 one can never fit
    probe_res, _, probe = _serve(reqs[:1], 1 << 34, 8)  # the server's own tables at 8 slots
    budget = int(probe["base_bytes"] + probe_res[0]["estimate"] + probe_res[0]["bytes"] // 2)
    res, xs, stats = _serve(reqs, budget, 8)
    assert stats["peak_bytes"] <= budget, (stats, budget)
    assert stats["estimate_misses"] == 0
    assert [r["status"] for r in res] == [fe.SOLVE_CONVERGED] * 4 + [fe.SOLVE_REFUSED]
    # each 40x40 request waited for the previous one's memory; the small one queued behind them
    assert res[1]["admitted_s"] >= res[0]["finished_s"]
    assert res[2]["admitted_s"] >= res[1]["finished_s"]
    assert res[3]["admitted_s"] >= res[2]["admitted_s"]
    for r in res[:4]:
        assert r["bytes"] <= r["estimate"]


def test_server_large_system_beside_small_ones(gpu):
    """A system above one wave of 512-row tiles (P1 720 x 720: 519,841 rows, over 512 rows per
    resident block on this GPU) iterates in the large-system engine on the high-priority stream,
    beside small ones in the other engine: every solution is bitwise the same as alone, and the large
    one meets the residual bound against the oracle's own system."""
    from paper_1501_01809_gb300 import fe
    sp = pytest.importorskip("scipy.sparse")
    specs = [(0.0, 720, 1, 1, 1), (0.0, 20, 2, 2, 1), (0.0005, 30, 1, 3, 2), (0.001, 64, 2, 1, 3),
             (0.002, 9, 1, 2, 2)]
    reqs = _requests(specs)
    res_mix, x_mix, stats = _serve(reqs, 1 << 34, 8)
    res_one, x_one, _ = _serve(reqs, 1 << 34, 1)
    assert stats["converged"] == len(reqs) and stats["estimate_misses"] == 0
    for i in range(len(reqs)):
        assert res_mix[i]["status"] == fe.SOLVE_CONVERGED and res_one[i]["status"] == fe.SOLVE_CONVERGED
        assert res_mix[i]["iters"] == res_one[i]["iters"], i
        np.testing.assert_array_equal(x_mix[i], x_one[i], err_msg=f"request {i}: mixed vs alone")
    r = reqs[0]
    rp, ci = O.sparsity(r["cmap"], r["cmap"], r["nn"], r["nn"])
    v, _ = O.assemble_mat(2, 1, O.LAPLACE, r["cmap"], r["mesh"].coords, r["mesh"].cell_vertex, rp, ci)
    b, _ = O.assemble_vec(2, 1, 1, r["cmap"], r["nn"], r["mesh"].coords, r["mesh"].cell_vertex, r["f"], r["cmap"])
    v, b = O.dirichlet_apply(rp, ci, v, b, r["bc"])
    A = sp.csr_matrix((v, ci, rp), shape=(r["nn"], r["nn"]))
    assert np.linalg.norm(b - A @ x_mix[0]) <= 1.5e-8 * np.linalg.norm(b)


def test_server_mesh_cache_skips_the_sparsity_build(gpu):
    """Requests that name the same mesh (mesh_key) share its device copy and sparsity: a cache hit
    builds no sparsity and copies no mesh, and the solutions are bitwise those of the same requests
    served without keys (every mesh built for its own request), mixed or one at a time."""
    from paper_1501_01809_gb300 import fe
    specs = [(0.0, 24, 2, 1, 2), (0.0, 10, 1, 3, 1), (0.001, 24, 2, 2, 1), (0.002, 17, 2, 4, 3),
             (0.002, 10, 1, 1, 1), (0.004, 24, 2, 3, 3)]
    keys = [7, 9, 7, 0, 9, 7]  # two shared meshes and one without a key
    reqs = _requests(specs)
    res_c, x_c, st_c = _serve(reqs, 1 << 34, 16, keys=keys)
    res_1, x_1, st_1 = _serve(reqs, 1 << 34, 1, keys=keys)
    res_n, x_n, st_n = _serve(reqs, 1 << 34, 16)
    for st in (st_c, st_1):
        assert st["converged"] == len(reqs) and st["estimate_misses"] == 0
        assert (st["sparsity_builds"], st["cache_misses"], st["cache_hits"]) == (3, 2, 3), st
    assert st_n["sparsity_builds"] == len(reqs) and st_n["cache_hits"] == 0
    for i in range(len(reqs)):
        assert res_c[i]["status"] == fe.SOLVE_CONVERGED
        np.testing.assert_array_equal(x_c[i], x_n[i], err_msg=f"request {i}: cached mesh vs its own")
        np.testing.assert_array_equal(x_c[i], x_1[i], err_msg=f"request {i}: mixed vs alone")
    # a hit holds only its own system: less than the request that built the mesh
    assert res_c[2]["bytes"] < res_c[0]["bytes"] + 1


def test_server_mesh_cache_evicts_under_the_budget(gpu):
    """With room for one mesh and one system, requests alternating between two meshes evict the
    unused cached mesh to admit the next one; every request converges within the budget."""
    from paper_1501_01809_gb300 import fe
    specs = [(0.0, 40, 2, 1, 1), (0.0, 41, 2, 2, 1), (0.0, 40, 2, 1, 2), (0.0, 41, 2, 2, 2)]
    reqs = _requests(specs)
    probe_res, _, probe = _serve(reqs[1:2], 1 << 34, 4)  # the server's own tables at 4 slots
    budget = int(probe["base_bytes"] + probe_res[0]["estimate"] + 4096)
    res, xs, st = _serve(reqs, budget, 4, keys=[1, 2, 1, 2])
    assert st["converged"] == len(reqs), st
    assert st["peak_bytes"] <= budget, (st, budget)
    assert st["cache_evictions"] >= 2 and st["sparsity_builds"] == 4, st
    ref, xr, _ = _serve(reqs, 1 << 34, 1)
    for a, b in zip(xs, xr):
        np.testing.assert_array_equal(a, b)
