"""Time the scatter surrogate's inference kernels on synthetic inputs.

    python -m paper_2002_12471_gb300.prof_mlp [--rows N] [--reps K] [--kernel 0|1|2]

Random He-initialised weights and standard-normal inputs; every repetition
is one lmosem_surrogate_infer call (BF16 weight preparation, input gather,
the network) timed with CUDA events; the network alone is read from the
library's per-kernel profile.  Prints one JSON line."""
import argparse
import json

import numpy as np

FLOPS_PER_ROW = 2 * (6 * 256 + 3 * 256 * 256 + 256)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", type=int, default=2_000_000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--kernel", type=int, default=0, help="0 automatic, 1 mma.sync chain, 2 tcgen05")
    args = ap.parse_args()
    import torch

    from . import lmosem as L
    from . import synthetic as S
    ph, g, *_ = S.workload("tiny16")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    rng = np.random.default_rng(1)
    blob = torch.from_numpy(L.surrogate_init(seed=2)).to(dev)
    X = torch.from_numpy(rng.standard_normal((args.rows, 6)).astype(np.float32)).to(dev)
    y = torch.empty(args.rows, dtype=torch.float32, device=dev)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream, profile=1, surrogate_kernel=args.kernel)
    try:
        L.lmosem_surrogate_infer(ctx, blob, X, y)   # warm-up
        L.lmosem_profile_read(ctx)
        ms = []
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.lmosem_surrogate_infer(ctx, blob, X, y)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        prof = L.lmosem_profile_read(ctx)
    finally:
        L.lmosem_destroy(ctx)
    mlp_ms = prof["mlp"][0] / args.reps
    print(json.dumps({"rows": args.rows, "kernel": args.kernel, "call_ms": float(np.mean(ms)),
                      "network_ms": mlp_ms, "network_tflops": args.rows * FLOPS_PER_ROW / (mlp_ms * 1e-3) / 1e12,
                      "finite": bool(torch.isfinite(y).all())}))


if __name__ == "__main__":
    main()
