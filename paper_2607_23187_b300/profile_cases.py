"""Small, bounded invocations of single kernels of the library, for profilers.

Each case builds a seeded synthetic problem, runs the steps before the
kernel of interest, then the kernel once with a bound on its work, and
prints one JSON line.  Meant to be run under ncu with ``-k`` and ``-c``:

    python -m paper_2607_23187_b300.profile_cases jacobi cfg2 1024 30000
        the Jacobi iteration (gap rule) on the preconditioned matrix,
        stopped after 30000 rotations
    python -m paper_2607_23187_b300.profile_cases lowprec cfg3 2048 2
        the low-precision eigenbasis with at most 2 FP32 sweeps per stage
    python -m paper_2607_23187_b300.profile_cases product 2048
        one split-BF16 product C = A^T B of order 2048
"""
import json
import sys
import time

import torch

import pjac_inputs as pin
from paper_2607_23187_b300 import pjac


def _jacobi(cfg: str, n: int, max_rot: int) -> dict:
    p = pin.config_problem(cfg, n=n)
    h = pjac.Handle()
    q, a1 = pjac.pjac_precondition(h, torch.tensor(p.a, device="cuda"))
    h.set_opts(max_rotations=max_rot)
    torch.cuda.synchronize()
    t = time.time()
    _, _, info, st = pjac.pjac_solve_preconditioned(h, a1, q, "gap", 1e-15, allow=(0, -4))
    torch.cuda.synchronize()
    el = time.time() - t
    h.close()
    return {"case": "jacobi", "cfg": cfg, "n": n, "rotations": info["rotations"], "status": st,
            "ms_jacobi": info["ms_jacobi"], "wall_s": el}


def _lowprec(cfg: str, n: int, sweeps: int) -> dict:
    p = pin.config_problem(cfg, n=n)
    h = pjac.Handle(fp32_sweeps=sweeps, transform="split_bf16")
    a = torch.tensor(p.a, device="cuda")
    torch.cuda.synchronize()
    t = time.time()
    pjac.pjac_eig_lowprec(h, a)
    torch.cuda.synchronize()
    el = time.time() - t
    d, r = h.fp32_sweeps_done()
    h.close()
    return {"case": "lowprec", "cfg": cfg, "n": n, "sweeps": [d, r], "wall_s": el}


def _product(n: int) -> dict:
    g = torch.Generator(device="cpu").manual_seed(n)
    a = torch.randn(n, n, dtype=torch.float64, generator=g).cuda()
    b = torch.randn(n, n, dtype=torch.float64, generator=g).cuda()
    h = pjac.Handle(transform="split_bf16")
    torch.cuda.synchronize()
    t = time.time()
    pjac.pjac_product(h, a, b, trans_a=True)
    torch.cuda.synchronize()
    el = time.time() - t
    h.close()
    return {"case": "product", "n": n, "wall_s": el}


def main(argv) -> int:
    pjac.load()
    what = argv[0]
    if what == "jacobi":
        r = _jacobi(argv[1], int(argv[2]), int(argv[3]))
    elif what == "lowprec":
        r = _lowprec(argv[1], int(argv[2]), int(argv[3]))
    elif what == "product":
        r = _product(int(argv[1]))
    else:
        raise SystemExit("unknown case %r" % what)
    print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
