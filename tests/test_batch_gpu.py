"""Batched stepping and the autotuner.

* every member of a batch advanced by one launch per step is bit-identical to
  the same domain stepped on its own (same storage type, same arithmetic);
* a member also matches the FP64 oracle;
* batches that cannot use the single launch fall back to one launch per member;
* tuning keeps the state and the results.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu
D2, D3 = inputs.D2Q9, inputs.D3Q19


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()


def _cases():
    sides, res, lids = inputs.batch_cavity_sides(6, seed=81)
    cases = [inputs.cavity2d(n, lid=v) for n, v in zip(sides, lids)]
    cases.append(inputs.random_case(D2, (136, 40), 0b11, seed=82, u_amp=0.05))
    cases.append(inputs.random_case(D2, (124, 33), 0b01, seed=83, u_amp=0.05, walls="mixed",
                                    force=(1e-4, -2e-4)))
    return cases


@pytest.mark.parametrize("precision", [M.F32, M.F64])
def test_batch_members_equal_standalone_runs(precision):
    cases = _cases()
    b = M.Batch.from_cases(cases, precision)
    info = b.info()
    assert info["members"] == len(cases) and info["launches_per_step"] == 1
    steps = 37                                 # one 32-step graph and 5 single launches
    b.step(steps)
    for m, case in zip(b.members, cases):
        s = M.Solver.from_case(case, precision)
        s.step(steps)
        assert np.array_equal(s.get_lattice_state(), m.get_lattice_state())
        assert m.params["steps"] == steps
        s.close()
    # and one member against the oracle
    case = cases[-1]
    r_g, u_g = b.members[-1].get_state()
    r_o, u_o = orc.step(D2, case.rho, case.u, case.periodic, wall=case.wall_mask, force=case.force,
                        nsteps=steps)
    tol = 1e-11 if precision == M.F64 else 2e-5
    assert np.sqrt(np.sum((u_g - u_o) ** 2) / np.sum(u_o ** 2)) < tol
    b.close()


def test_batch_fallback_and_3d():
    cases = [inputs.random_case(D3, (12, 10, 9), 0b000, seed=84, walls="box"),
             inputs.random_case(D3, (9, 8, 7), 0b111, seed=85)]
    b = M.Batch.from_cases(cases, M.F32)
    assert b.info()["launches_per_step"] == 2
    b.step(5)
    for m, case in zip(b.members, cases):
        s = M.Solver.from_case(case, M.F32)
        s.step(5)
        assert np.array_equal(s.get_lattice_state(), m.get_lattice_state())
        s.close()
    b.close()


def test_batch_rejects_mixed_lattices_and_foreign_steps():
    c2 = inputs.random_case(D2, (16, 16), 0b11, seed=86)
    c3 = inputs.random_case(D3, (8, 8, 8), 0b111, seed=87)
    cfg = lambda c: dict(lattice=c.lattice, dims=c.dims, dx=1.0, nu=1 / 6, periodic=c.periodic)
    with pytest.raises(M.MacLABError) as ei:
        M.Batch([cfg(c2), cfg(c3)])
    assert ei.value.status == M.ERR_INVALID
    b = M.Batch.from_cases([c2, c2])
    b.members[0].step(1)                       # stepped outside the batch
    with pytest.raises(M.MacLABError) as ei:
        b.step(1)
    assert ei.value.status == M.ERR_INVALID
    b.close()


def test_batch_tune_keeps_state():
    cases = _cases()
    b = M.Batch.from_cases(cases, M.F32)
    b.step(3)
    before = [m.get_lattice_state().copy() for m in b.members]
    rows = b.tune()
    assert rows in (2, 4, 8, 16, 32, 64)
    for m, x in zip(b.members, before):
        assert np.array_equal(m.get_lattice_state(), x)
    b.step(4)
    ref = M.Batch.from_cases(cases, M.F32)
    ref.step(7)
    for m, r in zip(b.members, ref.members):
        assert np.array_equal(m.get_lattice_state(), r.get_lattice_state())
    b.close()
    ref.close()


@pytest.mark.parametrize("lat,dims,periodic,walls", [(D3, (32, 24, 20), 0b000, "box"),
                                                     (D2, (64, 50), 0b01, "mixed")])
def test_single_domain_tune(lat, dims, periodic, walls):
    case = inputs.random_case(lat, dims, periodic, seed=88, walls=walls)
    s = M.Solver.from_case(case, M.F32)
    s.step(2)
    x = s.get_lattice_state().copy()
    ty, tz = s.tune()
    assert np.array_equal(s.get_lattice_state(), x)
    kernel = s.kernel_info()["kernel"]
    assert kernel in (M.KERNEL_TILED, M.KERNEL_FOLDED, M.KERNEL_SEGMENT, M.KERNEL_ROWS2, M.KERNEL_BLOCK)
    s.step(3)
    r_g, u_g = s.get_state()
    r_o, u_o = orc.step(lat, case.rho, case.u, periodic, wall=case.wall_mask, nsteps=5)
    assert np.sqrt(np.sum((u_g - u_o) ** 2) / np.sum(u_o ** 2)) < 1e-5
    # a second handle of the same shape takes the cached choice
    s2 = M.Solver.from_case(case, M.F32)
    assert s2.tune() == (ty, tz) and s2.kernel_info()["kernel"] == kernel
    s.close()
    s2.close()


def _depth_cases():
    """Members that exercise the two-step launch: a 28-quad segment boundary
    (nx = 136: segments of 28 and 6 quads), the narrowest rows (nx = 8, 12),
    every wall mode, periodic and closed axes, a force and a cavity."""
    sides, res, lids = inputs.batch_cavity_sides(3, seed=91)
    cases = [inputs.cavity2d(n, lid=v) for n, v in zip(sides, lids)]
    cases += [inputs.random_case(D2, (136, 40), 0b11, seed=92, u_amp=0.05),
              inputs.random_case(D2, (124, 33), 0b01, seed=93, u_amp=0.05, walls="mixed",
                                 force=(1e-4, -2e-4)),
              inputs.random_case(D2, (8, 11), 0b11, seed=94, u_amp=0.05),
              inputs.random_case(D2, (12, 9), 0b00, seed=95, u_amp=0.05, walls="box"),
              inputs.random_case(D2, (232, 17), 0b10, seed=96, u_amp=0.05, walls="mixed")]
    return cases


@pytest.mark.parametrize("precision", [M.F32, M.F64])
@pytest.mark.parametrize("steps,rows", [(1, 16), (2, 4), (7, 16), (37, 8), (64, 64)])
def test_two_steps_per_launch_bit_identical(precision, steps, rows):
    """Two updates per launch (temporal blocking) give the same bits as one
    update per launch: same sums in the same order, walls and closed
    boundaries reproduced in the intermediate rows."""
    cases = _depth_cases()
    ref = M.Batch.from_cases(cases, precision)
    ref.set_rows(rows)
    ref.step(steps)
    b = M.Batch.from_cases(cases, precision)
    b.set_rows(rows)
    b.set_depth(2)
    assert b.info()["steps_per_launch"] == 2
    b.step(steps)
    for m, r in zip(b.members, ref.members):
        assert np.array_equal(m.get_lattice_state(), r.get_lattice_state())
        assert m.params["steps"] == steps
    # the other buffer holds step n - 1 as after single steps: same residual
    for m, r in zip(b.members, ref.members):
        assert m.diagnostics()["residual"] == r.diagnostics()["residual"]
    b.close()
    ref.close()


def test_two_steps_per_launch_against_oracle():
    case = inputs.random_case(D2, (72, 29), 0b01, seed=97, u_amp=0.05, walls="mixed",
                              force=(2e-4, 1e-4))
    b = M.Batch.from_cases([case, case], M.F64)
    b.set_depth(2)
    b.step(9)
    r_g, u_g = b.members[0].get_state()
    r_o, u_o = orc.step(D2, case.rho, case.u, case.periodic, wall=case.wall_mask, force=case.force,
                        nsteps=9)
    assert np.abs(u_g - u_o).max() <= 1e-12 * np.abs(u_o).max()
    assert np.abs(r_g - r_o).max() <= 1e-12 * np.abs(r_o).max()
    b.close()


@pytest.mark.parametrize("kind", ["bf16", "narrow", "3d"])
def test_two_steps_per_launch_refused(kind):
    if kind == "bf16":
        b = M.Batch.from_cases(_cases()[:2], M.BF16_STORE)
    elif kind == "narrow":
        b = M.Batch.from_cases([inputs.random_case(D2, (4, 9), 0b11, seed=98),
                                inputs.random_case(D2, (16, 9), 0b11, seed=99)], M.F32)
    else:
        b = M.Batch.from_cases([inputs.random_case(D3, (8, 8, 8), 0b111, seed=100)], M.F32)
    with pytest.raises(M.MacLABError) as ei:
        b.set_depth(2)
    assert ei.value.status == M.ERR_UNSUPPORTED
    assert b.info()["steps_per_launch"] == 1
    b.step(3)
    b.close()


def test_batch_2d_fallback_with_a_non_interleaved_member():
    """A D2Q9 batch with a member whose nx is not a multiple of 4 steps one
    launch per member; the other members then use the tiled kernel (their
    default block or segment kernels take several steps per launch or need the
    single launch's work list) and still equal standalone runs bit for bit."""
    cases = [inputs.random_case(D2, (64, 40), 0b00, seed=86, walls="box"),
             inputs.random_case(D2, (30, 20), 0b11, seed=87),
             inputs.random_case(D2, (512, 300), 0b01, seed=88, walls="mixed")]
    b = M.Batch.from_cases(cases, M.F32)
    assert b.info()["launches_per_step"] == 3
    b.step(9)
    for m, case in zip(b.members, cases):
        s = M.Solver.from_case(case, M.F32)
        s.step(9)
        assert np.array_equal(s.get_lattice_state(), m.get_lattice_state())
        s.close()
    b.close()


@pytest.mark.parametrize("precision", [M.F32, M.F64])
@pytest.mark.parametrize("steps,rows", [(1, 16), (2, 4), (7, 16), (37, 8), (64, 2)])
def test_persistent_batch_bit_identical(precision, steps, rows):
    """Depth 3: every step pair of a call in one persistent cooperative launch
    over all members, blocks waiting only on the blocks next to their rows.
    Same sums in the same order as the two-step launches, so the same bits;
    the last step is a one-step launch, so the residual is the same too."""
    cases = _depth_cases()
    ref = M.Batch.from_cases(cases, precision)
    ref.set_rows(rows)
    ref.set_depth(2)
    ref.step(steps)
    b = M.Batch.from_cases(cases, precision)
    b.set_rows(rows)
    b.set_depth(3)
    assert b.info()["steps_per_launch"] == 3 and b.info()["rows"] == rows
    b.step(steps)
    b.sync()
    for m, r in zip(b.members, ref.members):
        assert np.array_equal(m.get_lattice_state(), r.get_lattice_state())
        assert m.params["steps"] == steps
    for m, r in zip(b.members, ref.members):
        assert m.diagnostics()["residual"] == r.diagnostics()["residual"]
    # a change of rows per item keeps the persistent form and the bits
    b.set_rows(2 * rows)
    ref.set_rows(2 * rows)
    b.step(9)
    ref.step(9)
    assert b.info()["steps_per_launch"] == 3
    for m, r in zip(b.members, ref.members):
        assert np.array_equal(m.get_lattice_state(), r.get_lattice_state())
    b.close()
    ref.close()


def test_persistent_batch_64_cavities_against_standalone_and_oracle():
    """The 64-cavity workload (sides 64..512, Re log-uniform in [100, 3200])
    in one persistent launch per call: every member equals its standalone run
    bit for bit after 301 steps, and the smallest one the FP64 oracle."""
    sides, res, lids = inputs.batch_cavity_sides(64, seed=4)
    cases = [inputs.cavity2d(n, lid=v) for n, v in zip(sides, lids)]
    b = M.Batch.from_cases(cases, M.F32)
    b.set_depth(3)
    steps = 301
    b.step(steps)
    b.sync()
    for i, (m, case) in enumerate(zip(b.members, cases)):
        if i % 8:
            continue  # every eighth member standalone (the bits of all are tied by the test above)
        s = M.Solver.from_case(case, M.F32)
        s.step(steps)
        assert np.array_equal(s.get_lattice_state(), m.get_lattice_state())
        s.close()
    k = int(np.argmin(sides))
    case = cases[k]
    r_g, u_g = b.members[k].get_state()
    r_o, u_o = orc.step(D2, case.rho, case.u, case.periodic, wall=case.wall_mask, nsteps=steps)
    assert np.sqrt(np.sum((u_g - u_o) ** 2) / np.sum(u_o ** 2)) < 1e-5
    b.close()


def test_persistent_batch_wait_runs_out():
    """A zero wait budget makes the first wait between blocks give up at once:
    the blocks end their sweeps, the next sync reports MACLAB_ERR_TIMEOUT once,
    and the context stays usable -- after set_state with the default budget
    the batch gives the two-step launches' bits."""
    cases = _depth_cases()
    b = M.Batch.from_cases(cases, M.F32)
    b.set_depth(3)
    b.set_wait_limit(0)
    b.step(10)
    with pytest.raises(M.MacLABError) as e:
        b.sync()
    assert e.value.status == M.ERR_TIMEOUT
    b.sync()  # the status word was cleared
    b.set_wait_limit(-1)
    for m, case in zip(b.members, cases):
        m.set_state(np.asarray(case.rho, np.float64), np.asarray(case.u, np.float64))  # e = 1
    b.step(10)
    b.sync()
    ref = M.Batch.from_cases(cases, M.F32)
    ref.set_depth(2)
    ref.step(10)
    for m, r in zip(b.members, ref.members):
        assert np.array_equal(m.get_lattice_state(), r.get_lattice_state())
    b.close()
    ref.close()


def test_persistent_batch_refused():
    for cases, precision in ((_cases()[:2], M.BF16_STORE),
                             ([inputs.random_case(D3, (8, 8, 8), 0b111, seed=100)], M.F32)):
        b = M.Batch.from_cases(cases, precision)
        with pytest.raises(M.MacLABError) as ei:
            b.set_depth(3)
        assert ei.value.status == M.ERR_UNSUPPORTED
        b.step(2)
        b.close()
