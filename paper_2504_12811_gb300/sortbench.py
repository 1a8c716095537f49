"""Time the radix sort entry point (aaag_radix_sort) on random keys.

python -m paper_2504_12811_gb300.sortbench [--keys N] [--bits B] [--reps R]

Sorts N uniform random keys (low B bits) with their indices as values, R
times after one warm-up call, and prints ms per sort and the bytes moved per
second (each pass reads and writes key and value, plus one histogram read).
"""
from __future__ import annotations

import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--keys", type=int, default=32 << 20)
    ap.add_argument("--bits", type=int, default=32)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    import torch
    from . import aaag
    dev = torch.device("cuda", 0)
    n, bits = args.keys, args.bits
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    k0 = torch.randint(0, 1 << min(bits, 31), (n,), device=dev, dtype=torch.int64, generator=g).to(torch.int32)
    v0 = torch.arange(n, device=dev, dtype=torch.int32)
    keys, vals = k0.clone(), v0.clone()
    ka, va = torch.empty_like(keys), torch.empty_like(vals)
    sb = aaag.aaag_radix_sort_scratch_bytes(n)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    st = aaag.current_stream()
    ms = []
    for rep in range(args.reps + 1):
        keys.copy_(k0)
        vals.copy_(v0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        alt = aaag.aaag_radix_sort(keys.data_ptr(), vals.data_ptr(), ka.data_ptr(), va.data_ptr(), n, bits,
                                   scratch.data_ptr(), sb, st)
        e1.record()
        torch.cuda.synchronize()
        if rep:
            ms.append(e0.elapsed_time(e1))
    out = ka if alt else keys
    ok = bool((out[1:].to(torch.int64) >= out[:-1].to(torch.int64)).all())
    passes = (bits + 7) // 8
    t = sum(ms) / len(ms)
    print(json.dumps({"keys": n, "key_bits": bits, "ms": t, "gbs": n * (16 * passes + 4) / (t / 1e3) / 1e9,
                      "sorted": ok}))
    if not ok:
        raise SystemExit("not sorted")


if __name__ == "__main__":
    main()
