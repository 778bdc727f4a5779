"""What the learned initialiser gains: the U-Net, trained briefly on the GPU
by the library's own forward and backward kernels on seeded pairs made with
the library's warp, predicts the initial field of held-out pairs (seeds never
used in training).  Each held-out pair is registered twice with the same
LNCC objective, from zero and from the prediction; the learned start must
reach the zero start's target (99 % of its decrease, the progress reading of
"equal final loss") in fewer iterations on the median pair, and fold
nowhere."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_trained_network_shortens_registration_on_held_out_pairs():
    from paper_2509_25044_gb300 import capi, experiments
    from paper_2509_25044_gb300.unet import UNet, training_pair
    capi.load()
    torch.manual_seed(0)
    n, n_train, epochs = 64, 256, 6
    net = UNet(n_in=n, seed=0, device=DEV)
    L = net.L
    data = []
    for i in range(n_train):
        p = training_pair(n, 20_000 + i, DEV)
        t = torch.empty((3, (n // 2) ** 3), device=DEV)
        capi.nn_check(L.reg_nn_field_down2(capi.ptr(p["v"]), capi.RegDims(n, n, n), capi.ptr(t), capi.stream_of(t)),
                      "field_down2")
        data.append((p["F"], p["M"], (float(p["F"].min()), float(p["F"].max())),
                     (float(p["M"].min()), float(p["M"].max())), t))
    rng = np.random.default_rng(0)
    first = last = None
    for ep in range(epochs):
        tot = torch.zeros((), dtype=torch.float64, device=DEV)
        for i in rng.permutation(n_train):
            F, M, fr, mr, t = data[i]
            net.pack(F, M, 1, fr, mr)
            net.forward()
            tot += net.loss_and_backward(t)[0]
            net.step(2e-4)
        mean = float(tot.item()) / n_train
        first = mean if first is None else first
        last = mean
    assert last < first, (first, last)
    assert capi.reg_get_device_error() == 0

    res = experiments.eval_init_pairs(net, n_pairs=8, n=n, seed0=95_000, iters=150, window=7, lam=2.0, lr=0.1)
    rows = [r for r in res["rows"] if r["zero"]["iters_to_target"] is not None]
    assert len(rows) >= 6, res
    # gain = zero-start iterations / learned-start iterations to the zero start's
    # target; a learned start that misses the target within the budget gains 0
    gains = [r["zero"]["iters_to_target"] / r["learned"]["iters_to_target"]
             if r["learned"]["iters_to_target"] is not None else 0.0 for r in rows]
    print("iterations-to-target gain per held-out pair:", [round(g, 2) for g in gains],
          "median", float(np.median(gains)))
    assert float(np.median(gains)) > 1.0, gains
    for r in res["rows"]:
        assert r["learned"]["fold"] == 0, r  # det(I + grad u) > 0 everywhere
