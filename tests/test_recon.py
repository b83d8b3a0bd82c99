"""Integration: the joint optimisation on the fetal-scale workload lowers the
loss and raises the PSNR of the Gaussian volume against the phantom."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_fetal_reconstruction_improves():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import inputs, recon
    case = inputs.fetal(0, init="flat")
    rec = recon.Reconstruction(case, n_sample=case["n_sample"], tile_h=12, tile_w=12)
    probe = recon.PSNRProbe(case["phantom"], case["N"])
    out = rec.run(200, probe=probe, eval_every=50)
    h = out["history"]
    print(h)
    losses = [x[2] for x in h[1:]]
    assert losses[-1] < 0.7 * losses[0]
    assert h[-1][3] > h[0][3] + 4.0
    assert all(h[k + 1][3] > h[k][3] for k in range(len(h) - 1))
    probe.close()
    rec.close()
