"""Small, self-contained launches of the library's kernels for profiler
captures (each holds a few GB of device memory at most).

  python -m paper_0809_4958_gb300.profile_cases batch [nboxes] [steps]
      a batch of uneven boxes drawn like the 512-box benchmark (E uniform in
      {24, 32, 48, 64}), FP32, velocity boundaries, stepped one step at a time
  python -m paper_0809_4958_gb300.profile_cases mlp_forward [boxes]
      three launches of the upsampler forward over the face rows of that many
      64^3 boxes (K = 16)
  python -m paper_0809_4958_gb300.profile_cases box [E] [storage] [steps]
      one box of E^3 sites (storage 0 FP64, 1 FP32, 2 binary16, 3 bfloat16
      deviations), velocity boundaries from random face samples, no chain,
      stepped one step at a time (256^3 binary16: 1.3 GB of populations)
  python -m paper_0809_4958_gb300.profile_cases step_interp [mlp|hermite] [boxes] [steps]
      that many 64^3 boxes (FP32, K = 16) stepped with the learned upsampler
      (random-init network) or with Hermite time interpolation alone
"""
from __future__ import annotations

import sys


def batch(nboxes: int = 96, steps: int = 12) -> None:
    import torch

    from . import inputs, lbtracer as lbt
    lbt.load()
    Es = [int(E) for E in inputs.batch_edges(0, nboxes, (24, 32, 48, 64))]
    tr = lbt.Tracers([lbt.box_desc(E, 0.8) for E in Es], lbt.LB_STORE_F32, stream=torch.cuda.Stream(), ring_slots=4)
    torch.cuda.synchronize()
    for b, E in enumerate(Es):
        tr.lb_init(b, torch.zeros((3, E, E, E), device="cuda"))
    gen = torch.Generator(device="cuda").manual_seed(0)
    nface = sum(18 * E * E for E in Es)
    faces = [torch.randn(nface, device="cuda", generator=gen) * 0.01 for _ in range(steps + 2)]
    for j in range(2):
        tr.lb_set_boundary(lbt.LB_ALL_BOXES, j, faces[j])
    for n in range(steps):
        tr.lb_set_boundary(lbt.LB_ALL_BOXES, n + 2, faces[n + 2])
        tr.lb_step(1)
    tr.lb_sync()
    print("batch", nboxes, "boxes", sum(E ** 3 for E in Es), "sites", steps, "steps")


def box(E: int = 256, storage: int = 2, steps: int = 8) -> None:
    import torch

    from . import lbtracer as lbt
    lbt.load()
    tr = lbt.Tracers([lbt.box_desc(E, 0.8)], storage, stream=torch.cuda.Stream(), ring_slots=4)
    torch.cuda.synchronize()
    tr.lb_init(0, torch.zeros((3, E, E, E), device="cuda", dtype=tr.real))
    gen = torch.Generator(device="cuda").manual_seed(0)
    faces = [(torch.randn(18 * E * E, device="cuda", generator=gen) * 0.01).to(tr.real) for _ in range(steps + 2)]
    tr.lb_set_boundary(0, 0, faces[0])
    for n in range(steps):
        tr.lb_set_boundary(0, n + 1, faces[n + 1])
        tr.lb_step(1)
    tr.lb_sync()
    print("box", E, "storage", storage, steps, "steps")


def mlp_forward(boxes: int = 256) -> None:
    import torch

    from . import inputs, lbtracer as lbt
    lbt.load()
    K, E = 16, 64
    rows = boxes * 6 * E * E
    params = lbt.Upsampler(K=K, batch_rows=1024, master=inputs.mlp_init(0, K)).export()
    gen = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn((rows, 32), device="cuda", generator=gen).to(torch.bfloat16)
    for _ in range(3):
        lbt.mlp_forward(params, K, X)
    torch.cuda.synchronize()
    print("mlp_forward", rows, "rows")


def step_interp(mode: str = "mlp", boxes: int = 64, steps: int = 32) -> None:
    import torch

    from . import inputs, lbtracer as lbt
    lbt.load()
    K, E = 16, 64
    ti = lbt.LB_TIME_MLP if mode == "mlp" else lbt.LB_TIME_HERMITE
    tr = lbt.Tracers([lbt.box_desc(E, 0.8, time_interp=ti, K=K) for _ in range(boxes)], lbt.LB_STORE_F32,
                     stream=torch.cuda.Stream(), ring_slots=4)
    torch.cuda.synchronize()
    for b in range(boxes):
        tr.lb_init(b, torch.zeros((3, E, E, E), device="cuda"))
    if ti == lbt.LB_TIME_MLP:
        params = lbt.Upsampler(K=K, batch_rows=1024, master=inputs.mlp_init(0, K)).export()
        tr.lb_mlp_bind(params, 0.05)
    gen = torch.Generator(device="cuda").manual_seed(0)
    nface = boxes * 18 * E * E
    nsamp = steps // K + 4
    faces = [torch.randn(nface, device="cuda", generator=gen) * 0.01 for _ in range(nsamp)]
    pushed = -1
    for n in range(steps):
        while pushed < n // K + 2:
            pushed += 1
            tr.lb_set_boundary(lbt.LB_ALL_BOXES, pushed, faces[pushed])
        tr.lb_step(1)
    tr.lb_sync()
    print("step_interp", mode, boxes, "boxes", steps, "steps")


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "batch"
    if case == "step_interp":
        mode = sys.argv[2] if len(sys.argv) > 2 else "mlp"
        step_interp(mode, *[int(a) for a in sys.argv[3:]])
    else:
        args = [int(a) for a in sys.argv[2:]]
        {"batch": batch, "mlp_forward": mlp_forward, "box": box}[case](*args)
