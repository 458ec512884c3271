"""Floating-point operations per cell-update of the method, per workload,
from the instrumented oracle (its own steps on a counting number type).

The oracle evaluates every stage at every cell (face fluxes of the phase
field included, where the GPU kernels skip them exactly), and collides each
population on its own, so these are the counts of the plain method.  Run on
crops of the workloads' initial states, one step:

    python oracle/count_flops.py
"""
import os
import sys

# the repository root, not this folder, first on the path (so that `oracle`
# is the package)
sys.path[0] = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

from oracle import oracle  # noqa: E402
from paper_2608_26908_gb300 import inputs  # noqa: E402

CROPS = {
    "dendrite2d": dict(nx=128, ny=128),
    "eutectic2d": dict(nx=256, ny=128),
    "dendrite3d": dict(nx=48, ny=48, nz=48),
    "eutectic3d": dict(nx=48, ny=48, nz=64),
    "adjoint2d": dict(nx=128, ny=128),
}


def main():
    for name, size in CROPS.items():
        sc = inputs.scenario(name, **size)
        phi, mu = inputs.initial_state(sc)
        f = oracle.rest_populations(sc)
        d = oracle.count_flops(sc, phi, mu, f, 1)
        print("%-11s %s  total %.0f" % (name, "  ".join("%s %.0f" % (k, v) for k, v in d.items() if k != "total"),
                                         d["total"]))


if __name__ == "__main__":
    main()
