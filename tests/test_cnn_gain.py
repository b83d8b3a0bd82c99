"""What the learned pose initialisation gains over the nominal start.

A small pose network is trained on the GPU (hand-written tensor-core
kernels) on slices that the library's own forward model renders from
synthetic Gaussian phantoms under random rigid motion U(+-20 deg) /
U(+-10 mm); on held-out slices rendered from phantoms of other seeds under
the same motion range, its predicted 6-DoF poses must be closer to the true
motion than the nominal (zero-motion) start the plain optimisation begins
from: the mean rotation error (angle of Rod(r_pred)^T Rod(r_true)) and the
mean translation error both below the nominal ones.  The full-size study
(2,000 phantoms, the reconstructions refined from either start) is
`python -m paper_2512_11624_b300.study learned`."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_trained_network_beats_nominal_pose():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import cnn
    torch.cuda.set_device(0)
    X, A, Y = cnn.make_training_set(400, motions_per_phantom=2, seed=3, max_deg=20.0, max_mm=10.0, workers=4)
    net = cnn.PoseNet(max_batch=256, seed=3)
    try:
        hist = cnn.train(net, X, A, Y, epochs=12, batch=256, lr=1e-3, seed=3)
        assert hist[-1][2] < 0.5 * hist[0][2], hist  # validation loss fell
        del X, A, Y
        Xv, Av, Yv = cnn.make_training_set(20, motions_per_phantom=1, seed=1003, max_deg=20.0, max_mm=10.0,
                                           workers=4)
        e = cnn.pose_errors_on_set(net, Xv, Av, Yv)
    finally:
        net.close()
    rot, rot0 = float(np.mean(e["net_rot_deg"])), float(np.mean(e["nominal_rot_deg"]))
    tr, tr0 = float(np.mean(e["net_trans_mm"])), float(np.mean(e["nominal_trans_mm"]))
    print("held-out slices %d: rotation %.2f deg (nominal %.2f), translation %.2f mm (nominal %.2f)" %
          (Xv.shape[0], rot, rot0, tr, tr0))
    assert Xv.shape[0] > 500
    assert rot < 0.95 * rot0, (rot, rot0)
    assert tr < 0.5 * tr0, (tr, tr0)
