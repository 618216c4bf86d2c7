"""Writes tests/golden/metric_psnr.txt: the PSNR (dB, whole image, against
the rasterised phantom) after each of the first 10 iterations of the damped
512 x 512 / 64-view solve (ellipse512_v64, seed 1000) with the prox-TV in the
(V^T V)^{-1} norm (Section 6.3; c_tv = 3, K = 20, damping 0.5 as in Section
7.2), computed by oracle.gamp alone.

    python tests/golden/make_metric_psnr.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def main():
    import numpy as np
    import synth
    from oracle import gamp, precond
    from oracle.geometry import Geometry
    c = synth.make_case("ellipse512_v64")
    g = Geometry(c["n"], c["n_views"], c["n_det"])
    curve = []

    def psnr(x):
        mu = precond.v_inverse(x, g)
        return 10 * np.log10(c["mu"].max() ** 2 / np.mean((mu - c["mu"]) ** 2))

    gamp.ct_solve(c["y"], c["I0"], g, 10, gamp.Options(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5, tv_metric=True),
                  on_iter=lambda t, x: curve.append(psnr(x)))
    with open(os.path.join(HERE, "metric_psnr.txt"), "w") as fh:
        fh.write("# PSNR (dB) after iterations 1..10 of the damped ellipse512_v64 solve with the\n")
        fh.write("# (V^T V)^-1-norm prox-TV (oracle); written by make_metric_psnr.py\n")
        fh.write(" ".join(repr(float(v)) for v in curve) + "\n")
    print(curve[-1])


if __name__ == "__main__":
    main()
