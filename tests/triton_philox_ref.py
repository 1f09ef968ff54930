"""Run Triton's own Philox4x32-10 (tl.philox) in its CPU interpreter.

Used by test_oracle_pins as an independent reference implementation.  Reads
counters (uint32 [n,4]) and a 64-bit seed from an .npz file, writes the four
output words next to it.  TRITON_INTERPRET must be set before triton loads.
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(c0p, c1p, c2p, c3p, o0, o1, o2, o3, seed, n: tl.constexpr):
    offs = tl.arange(0, n)
    c0 = tl.load(c0p + offs)
    c1 = tl.load(c1p + offs)
    c2 = tl.load(c2p + offs)
    c3 = tl.load(c3p + offs)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(o0 + offs, a)
    tl.store(o1 + offs, b)
    tl.store(o2 + offs, c)
    tl.store(o3 + offs, d)


def main(path):
    z = np.load(path)
    ctr = z["ctr"].astype(np.uint32)
    seed = int(z["seed"])
    n = ctr.shape[0]
    cs = [torch.from_numpy(ctr[:, i].view(np.int32).copy()) for i in range(4)]
    outs = [torch.empty(n, dtype=torch.int32) for _ in range(4)]
    s = seed if seed < 2**63 else seed - 2**64
    _philox_kernel[(1,)](*cs, *outs, s, n)
    out = np.stack([o.numpy().view(np.uint32) for o in outs], axis=1)
    np.save(path + ".out.npy", out)


if __name__ == "__main__":
    main(sys.argv[1])
