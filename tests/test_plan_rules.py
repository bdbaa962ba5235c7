"""Host logic of the launch plan (jac_resolve_plan, no GPU): the default
plans the library runs with on a 152-SM GB300, as the header and the design
notes state them and as the profiles and benchmarks were taken, and the
rejection of shapes the kernels lack."""
import pytest

from paper_2002_12115_gb300 import JacError
from paper_2002_12115_gb300.binding import KDEPTH_BALANCED, resolve_plan

SMS = 152


def plan(I, J, K, prec, **kw):
    p = resolve_plan(I, J, K, prec, sm_count=SMS, **kw)
    return p["tile_i"], p["tile_j"], p["kdepth"]


@pytest.mark.parametrize("dims,prec,want", [
    # FP32 / BF16: the smallest depth at which one round of CTAs holds every item
    ((129, 129, 257), "f32", (128, 8, 29)),        # 16 tiles x 9 k-blocks = 144 items
    ((129, 129, 257), "bf16", (128, 16, 14)),      # 16 warps: 8 tiles x 19 k-blocks = 152 items
    ((257, 257, 513), "f32", (128, 8, 256)),
    ((257, 257, 513), "bf16", (128, 16, 128)),
    # ... else shallow 8-plane items
    ((513, 513, 1025), "f32", (128, 8, 8)),
    ((513, 513, 1025), "bf16", (128, 16, 8)),
    # FP64: rounds x (kdepth + 3), or balanced ranges where those cost less
    ((129, 129, 257), "f64", (64, 8, KDEPTH_BALANCED)),
    ((513, 513, 1025), "f64", (64, 8, KDEPTH_BALANCED)),
    ((33, 33, 65), "f64", (32, 16, 1)),
    ((65, 65, 129), "f64", (64, 8, 7)),
])
def test_default_plans(dims, prec, want):
    assert plan(*dims, prec) == want


def test_one_round_rule_in_numbers():
    """FP32 129x129x257: items = 16 tiles x ceil(255 / kdepth) must fit 152
    CTAs; 29 is the smallest such depth (28 would need 160 items)."""
    tiles = ((129 - 2) // 128 + 1) * ((129 - 2 + 7) // 8)
    assert tiles * -(-255 // 29) <= SMS < tiles * -(-255 // 28)
    assert plan(129, 129, 257, "f32")[2] == 29


def test_explicit_entries_are_kept_and_the_rest_filled():
    assert plan(129, 129, 257, "f32", kdepth=5) == (128, 8, 5)
    assert plan(129, 129, 257, "f32", tile_j=16) == (64, 16, plan(129, 129, 257, "f32", tile_j=16)[2])
    assert plan(129, 129, 257, "f64", kdepth=KDEPTH_BALANCED)[2] == KDEPTH_BALANCED
    assert resolve_plan(129, 129, 257, "f32", sm_count=SMS, fuse=2)["fuse"] == 2
    assert resolve_plan(513, 513, 1025, "f32", sm_count=SMS, fuse=1)["fuse"] == 1


def test_two_sweep_passes_are_the_default_where_the_state_leaves_l2():
    """fuse = 0 resolves to two-sweep passes for FP32 storage whose two state
    buffers take more than half the L2 (128 MiB without a device), else to
    single sweeps; BF16-coefficient and FP64 storage never take passes."""
    def fuse(I, J, K, prec):
        return resolve_plan(I, J, K, prec, sm_count=SMS)["fuse"]
    assert fuse(513, 513, 1025, "f32") == 2          # 2.2 GB of state
    assert fuse(257, 257, 513, "f32") == 2           # 278 MB
    assert fuse(129, 129, 257, "f32") == 1           # 36 MB: stays in L2
    assert fuse(33, 33, 65, "f32") == 1
    # the boundary: 2 x pitch x J x K x 4 bytes against 64 MiB
    assert fuse(128, 256, 256, "f32") == 1           # exactly 64 MiB
    assert fuse(128, 256, 257, "f32") == 2           # 64.25 MiB
    for prec in ("bf16", "f64"):
        assert fuse(513, 513, 1025, prec) == 1


@pytest.mark.parametrize("kw", [dict(tile_j=5), dict(tile_i=48), dict(tile_j=16, tile_i=128),
                                dict(kdepth=-2), dict(fuse=3)])
def test_unsupported_plans_are_rejected(kw):
    with pytest.raises(JacError, match="JAC_EINVAL"):
        resolve_plan(129, 129, 257, "f32", sm_count=SMS, **kw)


def test_balanced_ranges_are_fp64_only():
    for prec in ("f32", "bf16"):
        with pytest.raises(JacError, match="JAC_EINVAL"):
            resolve_plan(129, 129, 257, prec, sm_count=SMS, kdepth=KDEPTH_BALANCED)


def test_bad_grids_are_rejected():
    with pytest.raises(JacError, match="JAC_EINVAL"):
        resolve_plan(2, 9, 9, "f32", sm_count=SMS)


def test_the_sm_count_moves_the_depth():
    """The one-round rule follows the SM count: with 76 SMs (one die) the
    129x129x257 FP32 items must be about twice as deep."""
    p = resolve_plan(129, 129, 257, "f32", sm_count=76)
    assert p["kdepth"] == 64      # 16 tiles x ceil(255 / 64) = 64 items <= 76
