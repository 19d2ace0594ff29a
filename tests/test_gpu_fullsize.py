"""FP64 parity at the bench's full size: the at-scale slab (1000 cells on
[-50, 50], 1e7 particles per step, moving-average filter, window ratio 5)
in the launch configuration the bench times, against the oracle run on the
same 1e7 particles.  Steps 1 and 2 have no splits; from step 3 on the
windows split particles (millions of daughters per step), so the splitting
lanes' own daughters, the record queue and the comb's multi-member groups
are all exercised at full size.  Bit-exact like the small parity cases:
counts, every fixed-point tally, closures, combed bank; LOSM solutions and
centers within 1e-12.  The oracle takes about 10-20 s per step here.
"""
import pytest

import workloads

pytestmark = pytest.mark.gpu

hww = pytest.importorskip("paper_2512_19925_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_parity import run_parity  # noqa: E402


def test_fp64_at_scale_full_size_parity():
    wl = workloads.plain_at_scale(particles_per_step=10_000_000, seed=1, precision="fp64")
    stats = run_parity(wl, 4)
    assert stats[0]["daughters"] == 0 and stats[2]["daughters"] > 1_000_000
    assert sum(s["segments"] for s in stats) > 8e7
