"""Train the learned hole inpainter on the GPU and write its weights file.

    python -m paper_2506_15183_gb300.weights.train [--frames 20000] [--tiles-per-frame 4]
        [--epochs 6] [--batch 64] [--out paper_2506_15183_gb300/weights/unet.yw]

Training set: seeded scenes rendered on the host (``scene.crop_config``: centred 512 x 512
crops of the 1832x1920 camera, fx = 916, the quest scene's statistics), the left eye
synthesized into the right by this library's plain path (``yoro_synthesize_zt``: the
warped colors, the hole mask, the warped depth), the network inputs of the frame's hole
tiles built on the device (``yoro_unet_prepare``), and the analytic ray-cast right eye as
ground truth.  Up to ``tiles_per_frame`` hole tiles per frame (drawn with a seeded
generator) stay on the device.  Training: ``yoro_unet_train_step`` (forward, loss on hole
pixels, backward, Adam), shuffled batches, the step size lowered to 0.3x and 0.1x after
60 % and 85 % of the steps.  At the end the hole PSNR of the network and of the paper's
fill against the ground truth on held-out crops is printed.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TRAIN_SEED0 = 100000  # training scenes; the benchmark's frames use seeds below 10000
EVAL_SEED0 = 900000   # held-out crops


def _render(seed):
    from paper_2506_15183_gb300 import scene

    cfg = scene.crop_config()
    (c, d, _), (cr, _, _) = scene.render_pair(cfg, seed, nthreads=1)
    return seed, c, d, cr


def _frames(seeds, workers):
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        yield from ex.map(_render, seeds, chunksize=8)


def _tiles_of(img, idx, ntx):
    """(len(idx), 64, 64, ...) tiles of an (H, W, ...) array at tile indices ty * ntx + tx."""
    return np.stack([img[64 * (i // ntx):64 * (i // ntx) + 64, 64 * (i % ntx):64 * (i % ntx) + 64] for i in idx])


def build_set(seeds, tiles_per_frame, workers, rng, keep_all=False):
    import torch

    import paper_2506_15183_gb300 as yoro
    from paper_2506_15183_gb300 import scene
    from paper_2506_15183_gb300 import unet as un
    from paper_2506_15183_gb300 import weights as W

    cfg = scene.crop_config()
    ntx = cfg.w // 64
    ntiles = ntx * (cfg.h // 64)
    hdl = yoro.yoro_create(**cfg.camera())
    prep = un.Inpainter(W.init_params(0), max_w=cfg.w, max_h=cfg.h)
    cap = len(seeds) * (ntiles if keep_all else tiles_per_frame)
    X = torch.empty((cap, 64, 64, 32), dtype=torch.bfloat16, device="cuda")
    GT = torch.empty((cap, 64, 64, 3), dtype=torch.uint8, device="cuda")
    HOLE = torch.empty((cap, 64, 64), dtype=torch.uint8, device="cuda")
    frames = []  # held-out evaluation keeps the frames
    xbuf = torch.empty((ntiles, 64, 64, 32), dtype=torch.bfloat16, device="cuda")
    rgba = torch.empty((cfg.h, cfg.w, 4), dtype=torch.uint8, device="cuda")
    mask = torch.empty((cfg.h, cfg.w), dtype=torch.uint8, device="cuda")
    zt = torch.empty((cfg.h, cfg.w), dtype=torch.float32, device="cuda")
    n = 0
    for seed, c, d, cr in _frames(seeds, workers):
        dg = torch.from_numpy(d).cuda()
        yoro.yoro_synthesize_zt(hdl, torch.from_numpy(c).cuda(), dg, rgba, mask, zt)
        idx = prep.prepare(rgba, mask, zt, dg, cfg.near, xbuf)
        if len(idx) == 0:
            continue
        pick = np.arange(len(idx)) if keep_all else np.sort(
            rng.choice(len(idx), size=min(tiles_per_frame, len(idx)), replace=False))
        sel = torch.from_numpy(pick).cuda()
        k = len(pick)
        X[n:n + k] = xbuf[sel]
        GT[n:n + k] = torch.from_numpy(np.ascontiguousarray(_tiles_of(cr[..., :3], idx[pick], ntx))).cuda()
        HOLE[n:n + k] = torch.from_numpy(np.ascontiguousarray(_tiles_of(mask.cpu().numpy(), idx[pick], ntx))).cuda()
        if keep_all:
            frames.append((seed, rgba.cpu().numpy().copy(), mask.cpu().numpy().copy(), zt.clone(), dg, cr))
        n += k
    yoro.yoro_destroy(hdl)
    prep.close()
    return X[:n], GT[:n], HOLE[:n], frames


def evaluate(params, frames):
    """Hole PSNR against the ground truth of the paper's fill and of the network, over the
    held-out frames (all hole pixels pooled)."""
    import torch

    from paper_2506_15183_gb300 import quality as Q
    from paper_2506_15183_gb300 import scene
    from paper_2506_15183_gb300 import unet as un

    cfg = scene.crop_config()
    net = un.Inpainter(params, max_w=cfg.w, max_h=cfg.h)
    se_plain = se_net = cnt = 0.0
    for _, plain, m, zt, dg, cr in frames:
        out = torch.from_numpy(plain).cuda()
        net.inpaint(out, torch.from_numpy(m).cuda(), zt, dg, cfg.near)
        got = out.cpu().numpy()
        h = m.astype(bool)
        se_plain += ((plain[h][:, :3].astype(float) - cr[h][:, :3]) ** 2).sum()
        se_net += ((got[h][:, :3].astype(float) - cr[h][:, :3]) ** 2).sum()
        cnt += 3 * h.sum()
    net.close()
    to_db = lambda se: 10 * np.log10(255.0 ** 2 / (se / cnt))
    return {"psnr_plain_fill": round(to_db(se_plain), 3), "psnr_network": round(to_db(se_net), 3),
            "hole_values": int(cnt), "frames": len(frames), "quality_module": Q.__name__}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=20000)
    ap.add_argument("--tiles-per-frame", type=int, default=4)
    ap.add_argument("--epochs", type=float, default=6.0)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--eval-frames", type=int, default=64)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--out", default=None)
    args = ap.parse_args()

    import torch

    from paper_2506_15183_gb300 import unet as un
    from paper_2506_15183_gb300 import weights as W

    torch.cuda.set_device(0)
    rng = np.random.default_rng(args.seed)
    t0 = time.time()
    X, GT, HOLE, _ = build_set(list(range(TRAIN_SEED0, TRAIN_SEED0 + args.frames)), args.tiles_per_frame,
                               args.workers, rng)
    _, _, _, held = build_set(list(range(EVAL_SEED0, EVAL_SEED0 + args.eval_frames)), 0, args.workers, rng,
                              keep_all=True)
    torch.cuda.synchronize()
    t_data = time.time() - t0
    N = X.shape[0]
    B = args.batch
    params = W.init_params(args.seed)
    before = evaluate(params, held)
    tr = un.Trainer(params, batch_tiles=B, lr=args.lr)
    steps = int(args.epochs * N / B)
    log = []
    t1 = time.time()
    order = torch.empty(0, dtype=torch.long, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(args.seed)
    pos = N
    for step in range(steps):
        if step == int(0.6 * steps):
            tr.set_lr(0.3 * args.lr)
        if step == int(0.85 * steps):
            tr.set_lr(0.1 * args.lr)
        if pos + B > N:
            order = torch.randperm(N, generator=g, device="cuda")
            pos = 0
        sel = order[pos:pos + B]
        pos += B
        tr.step(X[sel].contiguous(), GT[sel].contiguous(), HOLE[sel].contiguous())
        if step % 200 == 0 or step == steps - 1:
            loss = float(tr.read("loss")[0])
            log.append((step, round(loss, 6)))
            print(f"step {step}/{steps} loss {loss:.5f} ({time.time() - t1:.1f} s)", flush=True)
    if un.status() != 0:
        raise RuntimeError("inpainter kernel status")
    torch.cuda.synchronize()
    t_train = time.time() - t1
    trained = tr.read("params")
    final_loss = float(tr.read("loss")[0])
    tr.close()
    after = evaluate(trained, held)
    out = args.out or W.PATH
    W.save(trained, out, steps=steps, ktiles=(steps * B) // 1000, loss=final_loss, seed=args.seed)
    print(json.dumps({"frames": args.frames, "tiles": N, "batch": B, "steps": steps,
                      "data_s": round(t_data, 1), "train_s": round(t_train, 1),
                      "ms_per_step": round(1e3 * t_train / max(steps, 1), 3), "final_loss": final_loss,
                      "held_out_before": before, "held_out_after": after, "loss_log": log, "weights": out}),
          flush=True)


if __name__ == "__main__":
    main()
