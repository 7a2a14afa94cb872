"""Edge shapes through every reconstruction kernel, for the bounds-checked
build (run by tests/test_gpu_bounds.py in a process of its own with
DR_LIBRARY pointing at libdr_checked.so).

Each shape runs through the rows kernel, the per-pixel kernels (the
polynomial form, and the depth-table form by asking for the exact form), the
interval kernel, a persistent batch and the no-allocation entry point, and
the seeded random scans of every path kind through their plans' kernels in
core and streamed; after each, the plan's error word must be clear
(dr_plan_check raises with the device-source line of the first index found
out of range) and the result must match the FP64 oracle within the parity
tolerance.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def shapes():
    from tests.gen import synth
    from tests.golden.make_golden import odd_case

    odd, _ = odd_case()
    one = synth.tiny_scan(61, rows=1, cols=1, K=2)
    one.edges = np.array([-1.0, 1.0])                     # one pixel, two steps, one bin
    ragged = synth.tiny_scan(62, rows=3, cols=283, K=37)  # partial tiles, plain loads
    wide = synth.tiny_scan(63, rows=2, cols=280, K=300)   # several TMA chunks
    wide.edges = synth.bin_edges(-100.0, 350.0, 2.0)
    rot = synth.spot_scan(64, 5, 72, 29, 4, -60, 60, 0.7, rotate_deg=9.0, tilt_deg=3.0,
                          depth_range=(-0.03, 0.03))
    return [("tiny", synth.tiny_scan(60)), ("odd 6x9x4", odd), ("one pixel", one),
            ("ragged 283", ragged), ("wide K=300", wide), ("rotated", rot)]


def main():
    import torch

    from oracle import oracle as O
    from paper_2201_13309_gb300 import dr

    assert os.path.basename(dr.LIB_PATH) == "libdr_checked.so", dr.LIB_PATH

    def dev(images):
        return torch.from_numpy(np.ascontiguousarray(images).view(np.int16)).cuda()

    def close(got, sc, edge="leading"):
        ref = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges, edge)
        s = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)[None]
        err = np.abs(got.cpu().numpy().astype(np.float64) - ref)
        assert np.all(err <= 1e-4 * s), f"max err {(err / np.maximum(s, 1)).max()}"

    runs = 0
    jobs = []
    for name, sc in shapes():
        img = dev(sc.images)
        for kw in ({}, {"force_pixels": True}, {"force_pixels": True, "depth_form": "exact"},
                   {"force_intervals": True}, {"edge": "trailing"}):
            edge = kw.get("edge", "leading")
            plan = dr.Plan(sc.geom, sc.wires, sc.edges, **kw)
            out = plan.reconstruct(img)
            torch.cuda.synchronize()
            plan.check_device()
            close(out, sc, edge)
            runs += 1
            info = plan.info()
            if (sc.geom["cols"] % 8 == 0 and info["parts"] == 1
                    and (info["kernel"] != "rows" or info["pixels_per_thread"] == 4)):
                jobs.append((plan, img, torch.full_like(out, float("nan")), sc, edge))
    # seeded random scans of every path kind (tests/test_gpu_random_paths.py),
    # in core and streamed through two-row slabs into a pinned host output
    from tests.test_gpu_random_paths import random_scan
    ws = torch.empty(32 << 20, dtype=torch.uint8, device="cuda")
    for seed in range(24):
        sc, edge, _ = random_scan(seed)
        try:
            plan = dr.Plan(sc.geom, sc.wires, sc.edges, edge=edge)
        except dr.DrError:
            continue
        h_img = torch.from_numpy(np.ascontiguousarray(sc.images).view(np.int16)).pin_memory()
        out = plan.reconstruct(h_img.cuda())
        h_out = torch.full(tuple(out.shape), float("nan")).pin_memory()
        plan.reconstruct_streamed(h_img, h_out, ws, slab_rows=2)
        torch.cuda.synchronize()
        plan.check_device()
        close(out, sc, edge)
        close(h_out, sc, edge)
        runs += 1
    # one persistent batch over every job that it takes (rows, per-pixel and
    # interval tiles)
    batch = dr.Batch([(p, i, o) for p, i, o, _, _ in jobs])
    batch.launch()
    torch.cuda.synchronize()
    batch.check_device()
    for _, _, o, sc, edge in jobs:
        close(o, sc, edge)
    # the no-allocation entry point on the row-shared shapes
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for name, sc in shapes():
        if name == "rotated":
            continue
        out = torch.full((sc.B, sc.geom["rows"], sc.geom["cols"]), float("nan"), device="cuda")
        dr.reconstruct_rows_static(sc.geom, sc.wires, sc.edges, dev(sc.images), out, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0, (name, int(status.item()))
        close(out, sc)
    print(f"bounds-checked build: {runs} plans, {len(jobs)} batch jobs, clean")


if __name__ == "__main__":
    main()
