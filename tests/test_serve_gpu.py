"""The serving pattern: continuous batching of many design jobs on one GPU.
Each result must be the same alone and in the mix; admission must respect the
HBM cap (evicting idle meshes); the error paths must report, not hang."""
import numpy as np
import pytest
import torch

from paper_2505_02438_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def inputs(m, job, it):
    g = np.random.default_rng(1000 * job + it)
    rho = torch.as_tensor(g.uniform(0.001, 1.0, m.n_cells), device="cuda")
    u = torch.as_tensor(g.standard_normal(m.ndof), device="cuda")
    return rho, u


def run_mix(lib, jobs, iters, **server_kw):
    from paper_2505_02438_gb300.serve import Server
    meshes = {j["job"]: lib.Mesh.from_workload(j["workload"]) for j in jobs}
    srv = Server(**server_kw)
    tickets = []
    for it in range(iters):
        for j in jobs:
            m = meshes[j["job"]]
            rho, u = inputs(m, j["job"], it)
            vals = torch.empty(m.nnz, dtype=torch.float64, device="cuda")
            tickets.append((j["job"], it, rho, u, srv.submit(j["job"], j["workload"], rho, u, vals=vals)))
    results = [(job, it, rho, u, srv.wait(t)) for job, it, rho, u, t in tickets]
    stats = srv.stats()
    srv.close()
    return meshes, results, stats


def check_same_as_alone(meshes, results):
    for job, it, rho, u, r in results:
        assert r["status"] == 0, (job, it, r["status"])
        vals, dc, c = meshes[job].step(rho, u)
        # the same deterministic kernels: identical bits alone and in the mix
        assert torch.equal(vals, r["vals"]) and torch.equal(dc, r["dc"]) and torch.equal(c, r["c"]), (job, it)


def test_mix_matches_alone(lib):
    jobs = W.serving_stream(n_jobs=10, scale=0.2)
    meshes, results, stats = run_mix(lib, jobs, iters=3, max_slots=6, n_streams=4)
    check_same_as_alone(meshes, results)
    assert stats["completed"] == 30 and stats["failed"] == 0
    assert stats["mesh_setups"] == 10 and stats["evictions"] == 0
    assert sum(not r["mesh_was_resident"] for *_, r in results) == 10


def test_lowered_cap_evicts_idle_meshes(lib):
    jobs = W.serving_stream(n_jobs=8, scale=0.2)
    sizes = [lib.Mesh.from_workload(j["workload"]).device_bytes for j in jobs]
    cap = int(1.2 * max(sizes))
    meshes, results, stats = run_mix(lib, jobs, iters=2, hbm_cap_bytes=cap, max_slots=4, n_streams=2)
    check_same_as_alone(meshes, results)
    assert stats["evictions"] > 0
    assert stats["peak_resident_bytes"] <= cap


def _rectangles(nx, ny):
    coords, cells = W.structured_quad(nx, ny)
    coords = coords.copy()
    coords[:, 0] += 0.01 * coords[:, 0] ** 2
    return coords, cells


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_admission_bound_covers_each_built_mesh(lib, prec):
    """The bytes the server makes room for before building a job's mesh are at
    least what soptx_mesh_create allocates, on every assembly route."""
    from paper_2505_02438_gb300.serve import mesh_bytes_bound
    g = np.random.default_rng(5)
    cases = [("tri", 1, W.triangle_grid(60, 40, 0.2, g)), ("tri", 3, W.triangle_grid(40, 20, 0.2, g)),
             ("quad", 3, _rectangles(30, 20)), ("quad", 2, W.quad_grid(20, 10, 0.2, g)),
             ("tet", 2, W.kuhn_tets(6, 4, 4, 0.1, g)), ("hex", 1, W.structured_hex(20, 10, 10)),
             ("hex", 2, W.structured_hex(6, 4, 4)), ("hex", 3, W.hex_grid(3, 3, 2, 0.1, g))]
    for cell, k, (coords, cells) in cases:
        wl = W.Workload("bound", cell, k, coords, cells, elem_prec=prec)
        m = lib.Mesh.from_workload(wl)
        assert mesh_bytes_bound(wl) >= m.device_bytes, (cell, k, m.routes)
        m.close()


def test_error_paths(lib):
    from paper_2505_02438_gb300 import _native as N
    from paper_2505_02438_gb300.serve import Server
    wl = W.cantilever_hex(40, 20, 20)
    m = lib.Mesh.from_workload(wl)
    rho, u = inputs(m, 0, 0)
    # a mesh larger than the cap fails with ENOMEM
    srv = Server(hbm_cap_bytes=1 << 20)
    t = srv.submit(1, wl, rho, u)
    assert srv.wait(t)["status"] == 2
    with pytest.raises(N.SoptxError) as ei:
        srv.wait(12345)
    assert ei.value.code == 6
    srv.close()
    # a bounded wait that runs out reports ETIMEOUT and leaves the ticket valid
    srv = Server(max_queue=1)
    t = srv.submit(2, wl, rho, u)
    with pytest.raises(N.SoptxError) as ei:
        srv.wait(t, timeout_us=0)
    assert ei.value.code == 5
    # the queue holds one pending request while the first mesh is being set up
    busy = 0
    extra = []
    for k in range(3):
        try:
            extra.append(srv.submit(3 + k, wl, rho, u))
        except N.SoptxError as e:
            assert e.code == 4
            busy += 1
    assert srv.wait(t)["status"] == 0
    for x in extra:
        assert srv.wait(x)["status"] == 0
    assert busy >= 1
    srv.close()


def test_requests_of_different_jobs_are_in_flight_together(lib):
    """Requests of different jobs run on different streams: with their meshes
    resident and submitted together, their device intervals overlap (the
    record that shows it: gpu_start_us / gpu_end_us on one timeline), while
    the requests of one job run one after the other.  The meshes are as large
    as the serving mix's largest hexahedral ones (about 80 us of device work
    per request, several times the host's time to launch one): requests much
    shorter than a launch finish before the next one reaches the device."""
    from paper_2505_02438_gb300.serve import Server, overlap
    jobs = [dict(job=j, workload=W.cantilever_hex(100, 40, 40, wl=300 + j)) for j in range(3)]
    meshes = {j["job"]: lib.Mesh.from_workload(j["workload"]) for j in jobs}
    srv = Server(max_slots=8, n_streams=4)
    # first request per job makes its mesh resident
    warm = [srv.submit(j["job"], j["workload"], *inputs(meshes[j["job"]], j["job"], 0)) for j in jobs]
    assert all(srv.wait(t)["status"] == 0 for t in warm)
    # every input and output allocated first: a fresh device allocation synchronises
    # the device, which would serialise the requests
    reqs = []
    for it in range(3):
        for j in jobs:
            m = meshes[j["job"]]
            reqs.append((j, inputs(m, j["job"], it + 1), torch.empty(m.nnz, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    tickets = [(j["job"], srv.submit(j["job"], j["workload"], *x, vals=vals)) for j, x, vals in reqs]
    res = [(job, srv.wait(t)) for job, t in tickets]
    srv.close()
    assert all(r["status"] == 0 for _, r in res)
    for _, r in res:
        assert r["gpu_end_us"] > r["gpu_start_us"] >= 0.0
        assert abs((r["gpu_end_us"] - r["gpu_start_us"]) - r["gpu_us"]) <= 1.0 + 1e-3 * r["gpu_us"]
    ov = overlap([r for _, r in res])
    assert ov["max_in_flight"] >= 2, ov
    # one job's requests share its stream: they never overlap each other
    for j in jobs:
        iv = sorted((r["gpu_start_us"], r["gpu_end_us"]) for job, r in res if job == j["job"])
        assert all(b[0] >= a[1] - 1.0 for a, b in zip(iv, iv[1:])), iv


@pytest.mark.parametrize("group_small", [True, False])
def test_small_lattice_requests_share_grouped_launches(lib, group_small):
    """Requests on small Q4 and hex boxes admitted in one scheduler pass run as
    grouped launches (several requests per launch), with each result bitwise its
    mesh's own step; a larger hexahedral job in the mix takes the ordinary call."""
    jobs = [dict(job=j, workload=W.mbb_q4(8 + 7 * j, 4 + 3 * j, wl=400 + j)) for j in range(12)]
    jobs += [dict(job=50 + j, workload=W.cantilever_hex(6 + 4 * j, 4, 4, wl=450 + j)) for j in range(3)]
    jobs.append(dict(job=99, workload=W.cantilever_hex(30, 12, 12, wl=499)))
    meshes, results, stats = run_mix(lib, jobs, iters=3, max_slots=16, n_streams=4, group_small=group_small)
    check_same_as_alone(meshes, results)
    assert stats["completed"] == 48 and stats["failed"] == 0
    if group_small:
        assert 1 <= stats["groups"] < 45, stats
    else:
        assert stats["groups"] == 0
