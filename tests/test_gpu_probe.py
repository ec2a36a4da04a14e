"""The measurement probes of the benchmark: the FP64 FMA rate (the roofline peak),
the lane-FMA rate with part of every warp's lanes active, and the latency of a
dependent FMA."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_probes(mri):
    import torch
    scratch = torch.empty(152 * 8 * 256 * 4, dtype=torch.float64, device="cuda")
    props = torch.cuda.get_device_properties(0)
    full = mri.mri_probe_fp64_fma(scratch, iters=2048)
    assert full > 0
    lanes = {k: mri.mri_probe_fp64_lanes(scratch, k, iters=2048) for k in (32, 16, 8, 1)}
    # the lane-masked probe with every lane active measures the same pipe
    assert 0.8 * full <= lanes[32] <= 1.2 * full
    assert lanes[1] < lanes[8] < lanes[16] <= 1.05 * lanes[32]
    lat = mri.mri_probe_fp64_latency(scratch, iters=2048)
    assert 1.0 <= lat <= 1000.0
    print(f"{props.name}: {full / 1e9:.1f} GFMA/s; lane-FMA rates relative to 32 lanes: "
          + ", ".join(f"{k}: {lanes[k] / lanes[32]:.3f}" for k in (16, 8, 1)) + f"; dependent FMA {lat:.1f} cycles")
    with pytest.raises(mri.MriError):
        mri.mri_probe_fp64_lanes(scratch, 33)
