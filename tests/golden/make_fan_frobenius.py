"""Writes tests/golden/fan_frobenius.txt: ||Phi~||_F^2 (Algorithm 1, Steps 1
and 3; Phi~ = A V^-1, Eq. precondAMP_op) of the fan-beam workloads, computed
by oracle.fanbeam.frobenius_sq alone, one view per task across host
processes.  The 512 x 512 workload takes about 75,000 filtered ray images,
too many for a test to recompute; the GPU parity tests read the value here.

    python tests/golden/make_fan_frobenius.py
"""
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

NAMES = ("fan64_v30", "fan512_v102")


def _geom(name):
    import synth
    from oracle import fanbeam
    n, nv, nd, _ne, _rm, _rect, _I0, _it, sd, dd, ds = synth.FAN_CASES[name]
    return fanbeam.FanGeometry(n, nv, nd, sd, dd, ds)


def _view_term(args):
    name, k = args
    from oracle import fanbeam
    return fanbeam.frobenius_sq(_geom(name), views=[k])


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fan_frobenius.txt")
    lines = ["# ||Phi~||_F^2 of the fan-beam workloads (Phi~ = A V^-1, Eq. precondAMP_op),",
             "# summed over views in order by oracle.fanbeam.frobenius_sq; written by make_fan_frobenius.py",
             "# workload value"]
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count()) as pool:
        for name in NAMES:
            nv = _geom(name).n_views
            terms = pool.map(_view_term, [(name, k) for k in range(nv)])
            lines.append(f"{name} {sum(terms)!r}")
            print(lines[-1], flush=True)
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
