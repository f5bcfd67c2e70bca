"""The table of sweep launch shapes (host logic, no GPU): every shape fits the
kernel's tiling rules and one SM of a GB300, and the default comes first.  Shapes
whose warps each stay in one parity class get a queue of deferred comparisons per
warp and a table of their rows' neighbour offsets, where it costs no CTAs per SM;
the fused batch kernel's static arguments fit beside them."""
import pytest

SMEM_PER_SM = 228 * 1024      # shared memory per SM
SMEM_PER_CTA = 227 * 1024     # largest dynamic allocation of one CTA
RESERVED_PER_CTA = 1024       # shared memory the hardware keeps per resident CTA
GROUP_ARGS = 1024             # bound on the fused batch kernel's static shared memory (its sweep arguments)


@pytest.fixture(scope="module")
def pa():
    from paper_1711_02146_gb300 import build, pa as pa_mod
    build.build()
    return pa_mod


@pytest.mark.parametrize("L", [2, 4, 6, 8, 10, 12, 14, 16])
def test_shapes_follow_the_tiling_rules(pa, L):
    shapes = pa.sweep_shapes(L)
    assert shapes, "every supported size has a shape"
    N = L ** 3
    seen = set()
    for s in shapes:
        W, NT, MB = s["words"], s["threads"], s["ctas_per_sm"]
        assert s["L"] == L
        assert (W, NT, MB) not in seen
        seen.add((W, NT, MB))
        assert 32 % W == 0 and NT % W == 0 and NT <= 1024   # a partial last warp is allowed (L = 14)
        NP = NT // W                                   # row partitions
        assert NP % 2 == 0 and (L * L // 2) % (NP // 2) == 0
        assert 1024 % (32 * W) == 0                    # a tile never crosses the 1024-slot pitch unit
        tile = N * W * 4 + N * 32 + 33 * W * 4          # bit words, site records, slot table
        queues = (NT // 32) * 64 * 16                     # 64 deferred words of 16 bytes per warp
        rows = NP * (L * L // NP) * 8 * 4                 # per partition and row: 8 ints of offsets
        extra = queues + rows
        defer = NT % 32 == 0 and (NP // 2 * W) % 32 == 0 and MB * (tile + extra + RESERVED_PER_CTA) <= SMEM_PER_SM
        assert s["smem_bytes"] == tile + (extra if defer else 0)
        assert s["smem_bytes"] + GROUP_ARGS <= SMEM_PER_CTA
        assert MB * (s["smem_bytes"] + RESERVED_PER_CTA) <= SMEM_PER_SM
        if defer:
            assert MB * (s["smem_bytes"] + GROUP_ARGS + RESERVED_PER_CTA) <= SMEM_PER_SM
        assert MB * NT <= 2048


def test_unsupported_sizes_are_rejected(pa):
    for L in (0, 3, 18):
        with pytest.raises(pa.PAError):
            pa.sweep_shapes(L)
