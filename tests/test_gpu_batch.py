"""Independent instances in one context (batched solves): every instance of a
batch evolves exactly as it does alone (bitwise: per-row arithmetic and a
per-instance CFL step make it independent of its co-tenants), instances stop
at their own t_final, and the block-size autotuner neither changes results nor
leaves the state modified. Needs a GPU."""
import numpy as np
import pytest

from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _instances():
    out = [W.cylinder_instance(m, mach) for m, mach in ((8, 3.0), (11, 1.7), (6, 3.9))]
    v = W.vortex_workload(20)
    out.append((v.mesh, v.U0, None))
    box = M.structured_q1(9, 7, periodic_x=True, periodic_y=True)
    out.append((box, W.perturbed_state(box, 5, base=dict(rho=1.0, vel=(0.3, 0.1), p=1.0)), None))
    return out


def _solve(mesh, U0, bs, steps, precision, t_final=None, block=None):
    s = B.Solver(dim=mesh.dim, precision=precision)
    s.upload_mesh(mesh, bs)
    if block is not None:
        s.set_instances(block, t_final)
    s.set_state(U0)
    s.apply_boundary_conditions()
    for _ in range(steps):
        s.step(sync=False)
    return s.get_state(), s


@pytest.mark.parametrize("precision", [B.EH_PRECISION_FP64, B.EH_PRECISION_MIXED])
def test_batch_equals_instances_run_alone(precision):
    inst = _instances()
    mesh, off, bs = M.concatenate([m for m, _, _ in inst], [b for _, _, b in inst])
    U0 = np.concatenate([u for _, u, _ in inst], axis=1)
    Ub, sb = _solve(mesh, U0, bs, 6, precision, block=off)
    info = sb.instances()
    for k, (m, u, b) in enumerate(inst):
        Ua, sa = _solve(m, u, b, 6, precision)
        assert np.array_equal(Ub[:, off[k]:off[k + 1]], Ua), k
        assert info["last_dt"][k] == sa.diagnostics()["last_dt"]
    assert len(set(info["last_dt"].tolist())) == len(inst)  # each instance its own CFL step


def test_batch_instances_stop_at_their_final_time():
    inst = _instances()[:3]  # cylinders: slip nodes on the curved wall too
    mesh, off, bs = M.concatenate([m for m, _, _ in inst], [b for _, _, b in inst])
    U0 = np.concatenate([u for _, u, _ in inst], axis=1)
    t_final = np.array([0.02, 0.05, 0.5])
    s = B.Solver(dim=2)
    s.upload_mesh(mesh, bs)
    s.set_instances(off, t_final)
    s.set_state(U0)
    s.apply_boundary_conditions()
    for _ in range(40):
        s.step(sync=False)
    t = s.instances()["t"]
    assert t[0] == 0.02 and t[1] == 0.05 and t[2] < 0.5
    U1 = s.get_state()
    for _ in range(5):
        s.step()
    U2 = s.get_state()
    for k in (0, 1):  # frozen once finished, bit for bit
        assert np.array_equal(U1[:, off[k]:off[k + 1]], U2[:, off[k]:off[k + 1]])


def test_set_instances_rejects_coupled_rows():
    m = M.periodic_p1_square(8)
    s = B.Solver()
    s.upload_mesh(m)
    with pytest.raises(B.EulerError) as e:
        s.set_instances([0, 30, m.n])
    assert e.value.status == B.EH_ERR_BAD_MESH


def test_autotune_keeps_state_and_results():
    mesh, U0, bs = W.cylinder_problem(14)
    U0 = W.perturbed_state(mesh, 8)
    s = B.Solver()
    s.upload_mesh(mesh, bs)
    s.set_state(U0)
    s.apply_boundary_conditions()
    before = s.get_state()
    chosen = s.autotune(1)
    assert set(chosen[k] for k in chosen if k != "tau") <= {64, 128, 256}
    assert np.array_equal(s.get_state(), before)
    for _ in range(3):
        s.step(sync=False)
    ref, _ = _solve(mesh, U0, bs, 3, B.EH_PRECISION_FP64)
    assert np.array_equal(s.get_state(), ref)


@pytest.mark.parametrize("dim", [2, 3])
def test_launch_shapes_do_not_change_results(dim):
    """Rows per block and the cap on rows in flight per SM (grid-stride limiter
    kernels) change the schedule, never the arithmetic: bitwise equal states."""
    if dim == 2:
        mesh, U0, bs = W.cylinder_problem(14)
        U0 = W.perturbed_state(mesh, 8)
    else:
        mesh = M.structured_q1_3d(7, 6, 5, periodic=(True, True, True))
        U0 = W.perturbed_state(mesh, 9, base=dict(rho=1.0, vel=(0.4, 0.1, -0.2), p=1.0))
        bs = None
    ref, s = _solve(mesh, U0, bs, 3, B.EH_PRECISION_FP64)
    for tpb, cap in ((64, 0), (256, 0), (64, 256), (128, 512), (256, 2048)):
        q = B.Solver(dim=mesh.dim)
        q.upload_mesh(mesh, bs)
        for k in ("lim1", "pass", "final"):
            q.set_launch_shape(k, tpb, cap)
        q.set_launch_shape("visc", tpb)
        assert q.rows_per_sm()["pass"] == cap and q.block_sizes()["lim1"] == tpb
        q.set_state(U0)
        q.apply_boundary_conditions()
        for _ in range(3):
            q.step(sync=False)
        assert np.array_equal(q.get_state(), ref), (tpb, cap)
        q.close()


def test_launch_shape_rejects_bad_arguments():
    s = B.Solver(dim=2)
    for args in (("lim1", 96, 0), ("pass", 128, -1), ("pass", 128, 4096), ("visc", 128, 256), ("tau", 128, 0)):
        with pytest.raises(B.EulerError):
            s.set_launch_shape(*args)
    s.close()


def test_queued_line_searches_are_counted():
    """The limiter's line searches that the l = 1 check leaves open run in the
    queued kernels; the diagnostics count them (a flow with active limiting
    queues some; every iterated search was queued first)."""
    mesh, U0, bs = W.cylinder_problem(14)
    U0 = W.perturbed_state(mesh, 8)
    _, s = _solve(mesh, U0, bs, 4, B.EH_PRECISION_FP64)
    d = s.diagnostics()
    assert d["line_searches_deferred"] > 0
    assert 0 <= d["line_searches_iterated"] <= d["line_searches_deferred"]
    s.close()
