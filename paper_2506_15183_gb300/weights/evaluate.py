"""Hole quality of the learned inpainter and of the paper's fill on 1832x1920 frames.

    python -m paper_2506_15183_gb300.weights.evaluate [--frames 8] [--ssim-frames 4]

For seeds 1..frames of the 1832x1920 workload (200 primitives + ground, IPD 0.063 m):
the right eye synthesized by this library (yoro_synthesize_zt: the paper's fill), the
same frame with its holes repainted by the trained network (yoro_unet_inpaint, weights
from paper_2506_15183_gb300/weights/unet.yw), and the analytic ray-cast right eye as
ground truth.  Prints hole PSNR (all hole pixels of all frames pooled), and the mean
over frames of hole SSIM in the 11 x 11 Gaussian-window form and in the paper's
global-statistics form (quality.py), for the fill and the network against the ground
truth, and for the network against the fill.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=8)
    ap.add_argument("--ssim-frames", type=int, default=4)
    args = ap.parse_args()

    import torch

    import paper_2506_15183_gb300 as yoro
    from paper_2506_15183_gb300 import quality as Q
    from paper_2506_15183_gb300 import scene
    from paper_2506_15183_gb300 import unet as un
    from paper_2506_15183_gb300 import weights as W

    cfg = scene.quest_config()
    params, meta = W.read()
    net = un.Inpainter(params, max_w=cfg.w, max_h=cfg.h)
    hdl = yoro.yoro_create(**cfg.camera())
    rgba = torch.empty((cfg.h, cfg.w, 4), dtype=torch.uint8, device="cuda")
    mask = torch.empty((cfg.h, cfg.w), dtype=torch.uint8, device="cuda")
    zt = torch.empty((cfg.h, cfg.w), dtype=torch.float32, device="cuda")
    se = {"fill": 0.0, "net": 0.0}
    n = 0
    ssim = {k: [] for k in ("fill_gauss", "net_gauss", "fill_global", "net_global", "net_vs_fill_gauss")}
    holes = []
    for seed in range(1, args.frames + 1):
        (c, d, _), (gt, _, _) = scene.render_pair(cfg, seed)
        dg = torch.from_numpy(d).cuda()
        yoro.yoro_synthesize_zt(hdl, torch.from_numpy(c).cuda(), dg, rgba, mask, zt)
        fill = rgba.cpu().numpy()
        net.inpaint(rgba, mask, zt, dg, cfg.near)
        learned = rgba.cpu().numpy()
        m = mask.cpu().numpy().astype(bool)
        holes.append(float(m.mean()))
        for k, img in (("fill", fill), ("net", learned)):
            se[k] += ((img[m][:, :3].astype(np.float64) - gt[m][:, :3]) ** 2).sum()
        n += 3 * int(m.sum())
        if seed <= args.ssim_frames:
            ssim["fill_gauss"].append(Q.ssim_gaussian(fill, gt, m))
            ssim["net_gauss"].append(Q.ssim_gaussian(learned, gt, m))
            ssim["fill_global"].append(Q.ssim_global(fill, gt, m))
            ssim["net_global"].append(Q.ssim_global(learned, gt, m))
            ssim["net_vs_fill_gauss"].append(Q.ssim_gaussian(learned, fill, m))
    if un.status() != 0:
        raise RuntimeError("inpainter kernel status")
    db = lambda s: round(10 * np.log10(255.0 ** 2 / (s / n)), 3)  # noqa: E731
    print(json.dumps({
        "workload": f"1832x1920 quest frames, seeds 1-{args.frames} (hole pixels {np.mean(holes) * 100:.1f} %)",
        "weights": {"file": os.path.relpath(W.PATH, ROOT), **meta},
        "hole_psnr_db": {"paper_fill_vs_truth": db(se["fill"]), "network_vs_truth": db(se["net"])},
        "hole_ssim_gaussian": {"paper_fill_vs_truth": round(float(np.mean(ssim["fill_gauss"])), 4),
                               "network_vs_truth": round(float(np.mean(ssim["net_gauss"])), 4),
                               "network_vs_paper_fill": round(float(np.mean(ssim["net_vs_fill_gauss"])), 4)},
        "hole_ssim_global": {"paper_fill_vs_truth": round(float(np.mean(ssim["fill_global"])), 4),
                             "network_vs_truth": round(float(np.mean(ssim["net_global"])), 4)},
        "ssim_frames": args.ssim_frames,
    }), flush=True)
    yoro.yoro_destroy(hdl)
    net.close()


if __name__ == "__main__":
    main()
