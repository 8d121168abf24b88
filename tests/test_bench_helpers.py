"""The measurement arithmetic of bench.py (CPU only): the method's minimum
bytes per node and stage match their closed forms for the 2D (9-entry rows)
and 3D (27-entry rows) Q1 meshes, the planned per-kernel bytes follow their
per-unit figures, and the method-fixed FP64 count is a fixed function of the
mesh sizes (it does not depend on how the kernels evaluate the formulas)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("dim,row,per_node", [(2, 9, 328), (3, 27, 1064)])
def test_minimum_bytes_per_node_and_stage(bench, dim, row, per_node):
    # static edge data once (c_ij 8 dim, m_ij 8, col 4 B per entry), the state
    # read and written (2 x 8 S), m_i and row_ptr (8 + 4) per node
    n = 1000
    assert bench.survey_min_bytes_per_stage(n, row * n, dim) == per_node * n
    S = dim + 2
    assert per_node == row * (8 * dim + 8 + 4) + 2 * 8 * S + 12


def test_planned_bytes_of_the_viscosity_pass(bench):
    # 28 B per entry (col 4, c_ij 16, d_ij 8) and the state once per node (2D)
    n, nnz = 1000, 9000
    assert bench.survey_bytes("visc", n, nnz, 2) == 28 * nnz + 32 * n
    assert bench.survey_bytes("tau", n, nnz, 2) == 0


def test_method_fp64_count_is_linear_in_the_mesh_sizes(bench):
    # per node and per off-diagonal entry: doubling both doubles every count
    for k in ("prep", "visc", "low", "lim1", "pass", "final"):
        a = bench.method_fp64_flops(k, 1000, 9000, 2)
        b = bench.method_fp64_flops(k, 2000, 18000, 2)
        assert b == pytest.approx(2 * a) and a > 0
    # prep is per node only: d^2 + 9d + 25 operations
    assert bench.method_fp64_flops("prep", 1000, 9000, 2) == 1000 * (4 + 18 + 25)
