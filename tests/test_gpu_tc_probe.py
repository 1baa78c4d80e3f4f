"""The tensor-core probe of the p = 3 FR element operator (GPU).

bgk_probe_tc streams element-velocity panels through TMA tiled copies and
tcgen05 MMAs (BF16 hi/lo split, three products, FP32 accumulation in tensor
memory) and checks eight seeded panels against FP64 on the host.  The split
keeps 16 significant bits of the data, so an output's error stays within a
few 2^-16 of the sum of its terms' magnitudes; the tensor core truncates its
accumulation, so the outputs' magnitudes are shrunk slightly (a negative
bias) but far less than the split's own error."""
import pytest

pytestmark = pytest.mark.gpu


def test_fr_operator_on_tensor_cores_matches_fp64(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    r = bgk.probe_tc(16384)
    assert r["ms"] > 0 and r["flops"] > 0
    assert r["max_rel_err"] <= 6e-5, r
    assert abs(r["bias"]) <= 1e-5, r


def test_probe_rejects_bad_sizes(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    with pytest.raises(bgk.BGKError):
        bgk.probe_tc(8)
    with pytest.raises(bgk.BGKError):
        bgk.probe_tc(1 << 23)
