"""Runs Triton's own Philox4x32-10 (triton.language.philox) in Triton's CPU
interpreter and prints its outputs as JSON.  Used as an independent library
implementation that the oracle's Philox must reproduce bit for bit.

usage: TRITON_INTERPRET=1 python _triton_philox.py '<json {"ctr": [[c0,c1,c2,c3],...], "seed": S}>'
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _kernel(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0_ptr + i), tl.load(c1_ptr + i),
                           tl.load(c2_ptr + i), tl.load(c3_ptr + i))
    tl.store(out_ptr + i * 4 + 0, a)
    tl.store(out_ptr + i * 4 + 1, b)
    tl.store(out_ptr + i * 4 + 2, c)
    tl.store(out_ptr + i * 4 + 3, d)


def main():
    req = json.loads(sys.argv[1])
    ctr = np.asarray(req["ctr"], np.uint64).astype(np.uint32)
    n = ctr.shape[0]
    N = 1
    while N < n:
        N *= 2
    pad = np.zeros((N, 4), np.uint32)
    pad[:n] = ctr
    cols = [torch.from_numpy(pad[:, k].view(np.int32).copy()) for k in range(4)]
    out = torch.zeros(N * 4, dtype=torch.int32)
    _kernel[(1,)](out, cols[0], cols[1], cols[2], cols[3], int(req["seed"]), N=N)
    res = out.numpy().view(np.uint32).reshape(N, 4)[:n]
    print(json.dumps(res.astype(np.uint64).tolist()))


if __name__ == "__main__":
    main()
