"""Independent Philox4x32-10 reference for the oracle's generator (test helper).

Runs triton's own Philox (``tl.philox``) in triton's CPU interpreter and prints
the four output words for each (counter, key) read from stdin as JSON.  It is
run as a separate process because the interpreter must be selected before
triton is imported.  Used only by tests/test_oracle_philox.py.
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
def _philox_kernel(ctr_ptr, seed_ptr, out_ptr, n, BLOCK: tl.constexpr):
    i = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    m = i < n
    c0 = tl.load(ctr_ptr + 4 * i + 0, mask=m)
    c1 = tl.load(ctr_ptr + 4 * i + 1, mask=m)
    c2 = tl.load(ctr_ptr + 4 * i + 2, mask=m)
    c3 = tl.load(ctr_ptr + 4 * i + 3, mask=m)
    seed = tl.load(seed_ptr + i, mask=m)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 4 * i + 0, a, mask=m)
    tl.store(out_ptr + 4 * i + 1, b, mask=m)
    tl.store(out_ptr + 4 * i + 2, c, mask=m)
    tl.store(out_ptr + 4 * i + 3, d, mask=m)


def main():
    items = json.load(sys.stdin)
    n = len(items)
    ctr = np.array([it[:4] for it in items], dtype=np.uint32).view(np.int32).reshape(-1)
    seeds = np.array([it[4] | (it[5] << 32) for it in items], dtype=np.uint64).view(np.int64)
    out = torch.zeros(4 * n, dtype=torch.int32)
    BLOCK = 64
    _philox_kernel[((n + BLOCK - 1) // BLOCK,)](torch.from_numpy(ctr.copy()), torch.from_numpy(seeds.copy()),
                                                 out, n, BLOCK=BLOCK)
    res = out.numpy().view(np.uint32).reshape(n, 4).tolist()
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
