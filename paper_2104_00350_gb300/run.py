"""Run one of the synthetic workloads for a number of steps (a driver for profilers).

    python -m paper_2104_00350_gb300.run --case sphere --n 128 --steps 2 --precision fp32 [--explicit]

``--precision fp32_3xbf16`` runs the split-BF16 tensor-core z solve (3D cases, n = 128 or 256).

Cases: ``sphere`` (droplet on a sphere, n^3), ``porous`` (droplet over a sphere packing,
n^3), ``sinusoid`` (the six 512 x 256 sinusoidal-wall runs), ``ensemble`` (the 64-instance
2D ensemble).  ``--explicit`` selects the explicit Cahn-Hilliard variant (Eq. ExpCH).
The initial droplet is written, the step runs ``--steps`` times, and the status word and
the launch count are printed.
"""
from __future__ import annotations

import argparse
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=("sphere", "porous", "sinusoid", "ensemble"), default="sphere")
    ap.add_argument("--n", type=int, default=128, help="cells per axis (3D cases)")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--precision", choices=("fp32", "fp64", "fp32_3xbf16"), default="fp32",
                    help="fp32_3xbf16: the tensor-core z solve (3D, n = 128 or 256)")
    ap.add_argument("--explicit", action="store_true", help="explicit Cahn-Hilliard variant")
    args = ap.parse_args(argv)
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf
    from workloads import cases as W
    prec = {"fp64": ibpf.FP64, "fp32": ibpf.FP32, "fp32_3xbf16": ibpf.FP32_3XBF16}[args.precision]
    dt = np.float64 if prec == ibpf.FP64 else np.float32
    if args.case in ("sphere", "porous"):
        case = W.sphere_case(args.n) if args.case == "sphere" else W.porous_case(args.n)
        cl = [case]
    elif args.case == "sinusoid":
        cl = [W.sinusoid_wall_512x256(t, l) for t in (45.0, 90.0, 135.0) for l in (0.0, 0.01)]
    else:
        cl = W.ensemble_2d(64)
    if args.explicit:
        import dataclasses
        cl = [dataclasses.replace(c, params=dataclasses.replace(c.params, ch_scheme=1)) for c in cl]
    s = ibpf.solver_from_cases(cl, prec)
    s.precompute_weights()
    for k, c in enumerate(cl):
        if hasattr(c, "nz"):
            C0 = W.droplet_C3d(c, dt)
            s.write("C", C0, k)
            s.write("C_old", C0, k)
        else:
            s.write_state(W.initial_state(c), k)
    t0 = time.perf_counter()
    s.step(args.steps)
    status = max(s.query(ibpf.Q_STATUS, k) for k in range(len(cl)))
    print(f"case {args.case} precision {args.precision} steps {args.steps} status {status:g} "
          f"launches/step {s.query(ibpf.Q_LAUNCHES):g} wall {time.perf_counter() - t0:.3f} s")
    s.close()
    return 0 if status == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
