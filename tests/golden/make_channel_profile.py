"""Writes channel_512x256x256_profile.txt: the FP64 oracle's velocity
profile u_x(y) of the object-free 512x256x256 channel (walls at y = 0 and
y = 255, tau = 1, rho0 = 1, body force 1e-5 along x) after 20,000 steps,
from the fluid started at rest.  The flow is invariant along x and z, so a
2 x 256 x 2 column of the oracle carries it.  Only the oracle is run.

usage: python tests/golden/make_channel_profile.py [out]
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

NY, STEPS = 256, 20000


def profile():
    import oracle
    o = oracle.Oracle(2, NY, 2, walls=True, tau=1.0, rho0=1.0, body_force=(1e-5, 0.0, 0.0), friction=0.05)
    o.fluid_init()
    o.step(STEPS)
    return o.velocity()[0, 0, :, 0]


def main(out=os.path.join(HERE, "channel_512x256x256_profile.txt")):
    u = profile()
    with open(out, "w") as f:
        f.write("# FP64 oracle, object-free channel 512x256x256 (walls y=0,255), tau=1, rho0=1, body force 1e-5 "
                "along x, fluid at rest at step 0; u_x(y) after 20000 steps, y = 0..255 (written by "
                "tests/golden/make_channel_profile.py)\n")
        for v in u:
            f.write(f"{v:.17g}\n")


if __name__ == "__main__":
    main(*sys.argv[1:])
