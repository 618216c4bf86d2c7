"""Writes tests/golden/fan_psnr.txt: the PSNR (dB, over the whole image,
against the rasterised phantom) after each of the 30 iterations of the
damped fan-beam solve of fan512_v102 (Algorithm 1 with Phi~ = A V^-1, prox-TV
c_tv = 3, K = 20, damping 0.5 as in Section 7.2), computed by oracle.gamp
alone with the stored ||Phi~||_F^2 of fan_frobenius.txt.

    python tests/golden/make_fan_psnr.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def main():
    import numpy as np
    import synth
    from oracle import fanbeam, gamp, precond
    name = "fan512_v102"
    frob2 = None
    for line in open(os.path.join(HERE, "fan_frobenius.txt")):
        if line.startswith(name + " "):
            frob2 = float(line.split()[1])
    c = synth.make_case(name)
    f = c["fan"]
    g = fanbeam.FanGeometry(c["n"], c["n_views"], c["n_det"], f["src_dist"], f["det_dist"], f["det_spacing"])
    curve = []

    def psnr(x):
        mu = precond.v_inverse(x, g)
        return 10 * np.log10(c["mu"].max() ** 2 / np.mean((mu - c["mu"]) ** 2))

    gamp.ct_solve(c["y"], c["I0"], g, c["iters"], gamp.Options(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5),
                  frob2=frob2, on_iter=lambda t, x: curve.append(psnr(x)))
    with open(os.path.join(HERE, "fan_psnr.txt"), "w") as fh:
        fh.write("# PSNR (dB) after iterations 1..30 of the damped fan-beam solve of fan512_v102 (oracle);\n")
        fh.write("# written by make_fan_psnr.py\n")
        fh.write(" ".join(repr(float(v)) for v in curve) + "\n")
    print(curve[-1])


if __name__ == "__main__":
    main()
