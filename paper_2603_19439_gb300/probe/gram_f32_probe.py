"""Probe: three calls of grest_gram_f32 (C = X^T Y) on random FP32 blocks
X (1,000,000 x a) and Y (1,000,000 x b), for a profiler capture of the Gram
kernel that takes the shape.  Usage: python gram_f32_probe.py a b"""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import __graft_entry__  # noqa: E402
from paper_2603_19439_gb300 import grest as G  # noqa: E402
from paper_2603_19439_gb300 import workloads as wl  # noqa: E402

__graft_entry__.build()
torch.cuda.set_device(0)
a, b = int(sys.argv[1]), int(sys.argv[2])
n = 1_000_000
g, _ = wl.sbm_graph(200, 2, 0.1, 0.02, 71)  # a small context for its stream and scratch
rp, col, _ = g.csr()
tr = G.Tracker(g.n, rp, col, None, np.linalg.qr(np.random.default_rng(0).standard_normal((200, 4)))[0], np.ones(4), 4)
X = torch.randn(n, a, device="cuda")
Y = torch.randn(n, b, device="cuda")
C = torch.empty((a, b), dtype=torch.float64, device="cuda")
for _ in range(3):
    tr.gram_f32(X, Y, C)
torch.cuda.synchronize()
print("ok", C[0, 0].item())
tr.close()
