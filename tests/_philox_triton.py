"""Runs Triton's Philox4x32-10 (tl.philox) under its CPU interpreter on counters/keys read
from stdin (npz) and writes the outputs; executed as a subprocess with TRITON_INTERPRET=1."""
import sys

import numpy as np
import torch
import triton
import triton.language as tl


@triton.jit
def _k(c_ptr, out_ptr, seed_lo, seed_hi, N: tl.constexpr):
    offs = tl.arange(0, N)
    c0 = tl.load(c_ptr + offs * 4 + 0)
    c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2)
    c3 = tl.load(c_ptr + offs * 4 + 3)
    seed = (seed_hi.to(tl.uint64) << 32) | seed_lo.to(tl.uint64)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + offs * 4 + 0, a)
    tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c)
    tl.store(out_ptr + offs * 4 + 3, d)


def main(inp, outp):
    z = np.load(inp)
    ctr, keys = z["ctr"], z["keys"]          # [B, 64, 4] u32, [B, 2] u32
    outs = []
    for b in range(ctr.shape[0]):
        ct = torch.from_numpy(ctr[b].view(np.int32).copy())
        out = torch.zeros(ctr.shape[1] * 4, dtype=torch.int32)
        _k[(1,)](ct, out, int(keys[b, 0]), int(keys[b, 1]), N=ctr.shape[1])
        outs.append(out.numpy().view(np.uint32).reshape(-1, 4))
    np.save(outp, np.stack(outs))


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
