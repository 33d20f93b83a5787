"""Write the FP64 density-matrix AME ground-state population curves of the
8-qubit (N = 256) workload, for t_f = 10 and 100 ns, 2000-point grid.

Calls only the oracle (split-exact AME, Sec. II Eqs. ME2-H / ME2-L on the
symmetric split of the grid). Output: cfg_main_tf{10,100}_pgs.txt, one
population per grid point. Run: python tests/golden/make_cfg_main_ame.py [t_f ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import ame  # noqa: E402


def main():
    tfs = [float(a) for a in sys.argv[1:]] or [10.0, 100.0]
    for tf in tfs:
        inst = W.cfg_main(t_f=tf)
        t = time.time()
        out = ame.run(inst)
        path = os.path.join(HERE, f"cfg_main_tf{tf:g}_pgs.txt")
        np.savetxt(path, out["p_gs"], fmt="%.15e",
                   header=f"ground-manifold population, 8-qubit TFIM workload, t_f = {tf:g} ns, "
                          f"2000-point grid, split-exact FP64 AME ({time.time() - t:.0f} s)")
        print(path, out["p_gs"][-1], time.time() - t, flush=True)


if __name__ == "__main__":
    main()
