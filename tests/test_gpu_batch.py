"""Batched 2D boxes (lbm_batch_*) against unbatched handles and the FP64 oracle.

A batch member runs the same per-node step as a single box, so every member must equal, bit for
bit, an unbatched handle created with the same arguments, whatever the tile shape, the CTAs per
SM or the CUDA-graph length; the FP64 oracle pins the arithmetic itself (populations within 1e-12
after 100 steps, the bound of the single-box parity tests).
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_09041_gb300 import lbm as L  # noqa: E402

# uneven members: ragged tiles in x and y, a box narrower than one warp, mixed wall sets
SIZES = [(37, 19), (64, 64), (100, 33), (17, 80), (96, 128), (8, 6)]
RA = [1e3, 1e5, 3e4, 1e6, 2e4, 1e4]
PR = [0.71, 7.0, 1.3, 0.71, 4.0, 2.0]


def member_walls(k):
    if k % 3 == 2:
        return L.Walls.rayleigh_benard(seed=100 + k, perturb=1e-3)
    return L.Walls.cavity(2)


def oracle_walls(k):
    if k % 3 == 2:
        return O.rayleigh_benard_bc(seed=100 + k, perturb=1e-3)
    return O.cavity_bc(2)


def make_batch(precision="fp32", sizes=SIZES, Ra=RA, Pr=PR, walls=None):
    walls = walls or [member_walls(k) for k in range(len(sizes))]
    return L.Batch(sizes, Ra, Pr, Ma=0.1, walls=walls, precision=precision)


def single(k, precision="fp32", sizes=SIZES, Ra=RA, Pr=PR, walls=None):
    w = (walls or [member_walls(j) for j in range(len(sizes))])[k]
    nx, ny = sizes[k]
    return L.Lattice("d2q9", nx, ny, 1, Ra=Ra[k], Pr=Pr[k], Ma=0.1, walls=w, precision=precision)


def perturb_members(b, seed):
    """Give every member a seeded non-equilibrium state (same for the unbatched runs)."""
    states = []
    for k in range(b.count):
        f, g = b.get_populations(k)
        f = synth.perturbed(f, seed + 2 * k, 0.05)
        g = synth.perturbed(g, seed + 2 * k + 1, 0.05)
        b.set_populations(k, f, g)
        states.append((f, g))
    return states


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_members_equal_unbatched_runs_bitwise(precision):
    b = make_batch(precision)
    states = perturb_members(b, 10)
    b.step(70)                       # two graph replays of 32 steps and 6 plain launches
    flags = b.sync()
    assert not flags.any()
    for k in range(b.count):
        lat = single(k, precision)
        lat.set_populations(*states[k])
        lat.step(70)
        lat.sync()
        fb, gb = b.get_populations(k)
        fs, gs = lat.get_populations()
        assert np.array_equal(fb, fs) and np.array_equal(gb, gs), f"member {k} {SIZES[k]}"
        lat.close()
    b.close()


def test_fp64_members_match_oracle():
    b = make_batch("fp64")
    picks = (0, 2, 5)
    oracles = {}
    for k in picks:
        nx, ny = SIZES[k]
        ora = O.Oracle(2, nx, ny, 1, bc=oracle_walls(k), Ra=RA[k], Pr=PR[k], Ma=0.1)
        f, g = ora.get_state()
        f = synth.perturbed(f, 40 + k, 0.05)
        g = synth.perturbed(g, 41 + k, 0.05)
        ora.set_state(f, g)
        b.set_populations(k, f, g)
        oracles[k] = ora
    b.step(100)
    for k in picks:
        oracles[k].step(100)
        fb, gb = b.get_populations(k)
        fo, go = oracles[k].get_state()
        err = max(np.abs(fb - fo).max(), np.abs(gb - go).max())
        assert err <= 1e-12, (k, err)
    b.close()


@pytest.mark.parametrize("shape", [(32, 1, 2), (32, 4, 8), (64, 1, 16), (128, 2, 4), (256, 1, 8),
                                   (64, 2, 0)])
def test_launch_shape_does_not_change_results(shape):
    ref = make_batch("fp32")
    states = perturb_members(ref, 20)
    ref.step(40)
    b = make_batch("fp32")
    for k, (f, g) in enumerate(states):
        b.set_populations(k, f, g)
    b.set_launch(*shape, graph_steps=8)
    b.step(40)
    inf = b.info()
    assert (inf.tile_x, inf.tile_y, inf.graph_steps) == (*shape[:2], 8)
    assert inf.ctas_per_sm == shape[2] or (shape[2] == 0 and inf.ctas_per_sm >= 1)
    for k in range(b.count):
        fa, ga = ref.get_populations(k)
        fb, gb = b.get_populations(k)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), k
    ref.close()
    b.close()


def test_graph_replay_equals_plain_launches():
    a, b = make_batch("fp32"), make_batch("fp32")
    states = perturb_members(a, 30)
    for k, (f, g) in enumerate(states):
        b.set_populations(k, f, g)
    b.set_launch(64, 2, 8, graph_steps=0)
    a.step(96)
    b.step(96)
    assert a.info().steps == b.info().steps == 96
    for k in range(a.count):
        fa, ga = a.get_populations(k)
        fb, gb = b.get_populations(k)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), k
    a.close()
    b.close()


def test_autotuner_keeps_state_and_picks_a_valid_shape():
    b = make_batch("fp32")
    perturb_members(b, 50)
    b.step(3)
    before = [b.get_populations(k) for k in range(b.count)]
    tx, ty, cps = b.tune(4)
    inf = b.info()
    assert (inf.tile_x, inf.tile_y, inf.ctas_per_sm) == (tx, ty, cps)
    assert tx in (32, 64, 128, 256) and tx * ty <= 256 and 1 <= cps <= 1024
    assert inf.steps == 3
    for k in range(b.count):
        f, g = b.get_populations(k)
        assert np.array_equal(f, before[k][0]) and np.array_equal(g, before[k][1]), k
    assert not b.sync().any()
    b.close()


def test_nusselt_of_a_member_equals_unbatched():
    b = make_batch("fp32")
    b.step(200)
    for k in (0, 1, 4):
        lat = single(k, "fp32")
        lat.step(200)
        assert b.nusselt(k, 0) == lat.nusselt(0)
        assert b.nusselt(k, 1) == lat.nusselt(1)
        lat.close()
    # member 2 is a Rayleigh-Benard box: its fixed-T faces are -y and +y
    lat = single(2, "fp32")
    lat.step(200)
    assert b.nusselt(2, 2) == lat.nusselt(2)
    with pytest.raises(L.LbmError):
        b.nusselt(2, 0)             # periodic face
    with pytest.raises(L.LbmError):
        b.nusselt(len(SIZES), 0)    # no such member
    lat.close()
    b.close()


def test_divergence_is_flagged_per_member():
    b = make_batch("fp32")
    states = perturb_members(b, 60)
    f, g = states[3]
    b.set_populations(3, -np.abs(f), g)        # negative density everywhere in member 3
    b.step(5)
    flags = b.sync()
    assert flags.tolist() == [0, 0, 0, 1, 0, 0]
    # the other members are untouched by member 3's failure
    for k in (0, 4):
        lat = single(k, "fp32")
        lat.set_populations(*states[k])
        lat.step(5)
        fb, _ = b.get_populations(k)
        fs, _ = lat.get_populations()
        assert np.array_equal(fb, fs)
        lat.close()
    b.close()


def test_invalid_launch_shapes_are_rejected():
    b = make_batch("fp32")
    for bad in [(48, 2, 8), (64, 8, 8), (256, 1, 1025), (64, 2, -1)]:
        with pytest.raises(L.LbmError):
            b.set_launch(*bad)
    with pytest.raises(L.LbmError):
        b.step(-1)
    b.close()


def test_ensemble_workload_members_equal_unbatched():
    """The 64-cavity ensemble (sides 64..512, Ra 1e3..1e7, Pr 0.71..7), FP32, autotuned: sampled
    members equal their unbatched runs bit for bit, and the divergence flags agree with the
    unbatched runs' status."""
    sizes, Ra, Pr = synth.ensemble_2d()
    b = L.Batch(sizes, Ra, Pr, Ma=0.1, precision="fp32")
    b.tune(5)
    b.step(300)
    flags = b.sync()
    assert b.info().total_nodes == sum(x * y for x, y in sizes)
    order = np.argsort([x * y for x, y in sizes])
    picks = {int(order[0]), int(order[len(order) // 2]), int(order[-1]), int(np.argmax(Ra))}
    for k in sorted(picks):
        nx, ny = sizes[k]
        lat = L.Lattice("d2q9", nx, ny, 1, Ra=Ra[k], Pr=Pr[k], Ma=0.1, precision="fp32")
        lat.step(300)
        try:
            lat.sync()
            diverged = 0
        except L.LbmError as e:
            assert e.status == L.LBM_EDIVERGED
            diverged = 1
        assert flags[k] == diverged, k
        if not diverged:
            fb, gb = b.get_populations(k)
            fs, gs = lat.get_populations()
            assert np.array_equal(fb, fs) and np.array_equal(gb, gs), k
        lat.close()
    b.close()
