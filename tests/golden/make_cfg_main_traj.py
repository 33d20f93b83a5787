"""Write oracle trajectories of the 8-qubit (N = 256) workload at full size
(t_f = 10 ns, 2000-point grid, trajectory stream seed of the workload) for a
few trajectory indices, so that GPU runs of all 10^4 trajectories can be
checked trajectory by trajectory on those samples.

Calls only the oracle (serial waiting-time sampler, Sec. IV). Output:
cfg_main_tf10_traj.json with, per sampled trajectory, its jump records and
its ground-manifold population at every 100th grid point and at s = 1.
Run: python tests/golden/make_cfg_main_traj.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import trajectories  # noqa: E402

SAMPLES = [0, 1, 2, 3, 4, 5, 6, 7, 4999, 9999]


def main():
    inst = W.cfg_main(t_f=10.0)
    t = time.time()
    p, jumps, _ = trajectories.sample(inst, SAMPLES)
    out = {"t_f": inst.t_f, "n_grid": inst.n_grid, "seed": inst.seed, "samples": SAMPLES,
           "p_gs_every_100": {str(tr): [float(x) for x in p[i, ::100]] + [float(p[i, -1])]
                              for i, tr in enumerate(SAMPLES)},
           "jumps": [{k: (float(v) if isinstance(v, float) else int(v)) for k, v in j.items()} for j in jumps],
           "seconds": time.time() - t}
    with open(os.path.join(HERE, "cfg_main_tf10_traj.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(len(jumps), "jumps", time.time() - t, flush=True)


if __name__ == "__main__":
    main()
