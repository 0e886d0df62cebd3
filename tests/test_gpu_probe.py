"""The throughput probe behind the reported rooflines (xyz_probe_peaks):
positive rates in the ratios of the instruction classes it measures (32-bit
adds issue at least as fast as lop3, and lop3 faster than popc), an SM clock
within the device's range, and the device's SM count."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_peaks_are_plausible():
    import torch

    from paper_1610_05108_gb300 import build, xyz
    build.build()
    xyz.load()
    pk = xyz.probe_peaks()
    props = torch.cuda.get_device_properties(0)
    assert pk["sms"] == props.multi_processor_count
    assert 200.0 < pk["sm_mhz"] < 3000.0
    for k in ("alu_ops_per_s", "iadd_ops_per_s", "popc_ops_per_s"):
        assert pk[k] > 1e11, (k, pk)
    assert pk["iadd_ops_per_s"] >= 0.9 * pk["alu_ops_per_s"]
    assert pk["alu_ops_per_s"] > 1.5 * pk["popc_ops_per_s"]
    # per SM and clock: at most one warp instruction per scheduler, 4 per SM
    per_clk = pk["iadd_ops_per_s"] / (pk["sms"] * pk["sm_mhz"] * 1e6)
    assert per_clk <= 4 * 32 * 1.05
