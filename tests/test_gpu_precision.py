"""Storage precision on the 512x256x256 channel (33.5 M cells, walls in y,
tau = 1, body force 1e-5, object-free), 20,000 steps: the velocity field of
FP32, FP16-shifted and BF16-shifted storage against the FP64 oracle's
same-step profile, and the drift of the total mass (FP64 reduction).

The oracle runs a 2 x 256 x 2 column of the same channel: without objects
the flow is invariant along x and z (pinned in test_oracle_fluid), so every
column of the full box carries the oracle's FP64 profile.  At 20,000 steps
the start-up is not finished (relaxation time H^2 / (pi^2 nu) ~ 39,000
steps), so the comparison is at the same step, not with the steady state.
Bars: FP32 1e-5 (the fluid parity bar; measured 6.9e-6), FP16-shifted
1e-3 (the bar the 16-bit form is held to), BF16-shifted 2e-2 (its 8-bit
mantissa).  The FP32 collision is the increment form (fluid_core.cuh), so
FP32 storage carries no systematic per-step error; the earlier direct form
made nearly the same rounding error in a cell every step (the constant 1/6
rounded, the force added into the momentum before rounding) and reached
4.3e-4 here.
"""
import numpy as np
import pytest

import oracle
from paper_1312_3426_gb300 import lbib

pytestmark = pytest.mark.gpu

NX, NY, NZ, STEPS = 512, 256, 256, 20000


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_3426_gb300 import build
    build.build()
    lbib.load()


@pytest.fixture(scope="module")
def profile():
    o = oracle.Oracle(2, NY, 2, walls=True, tau=1.0, rho0=1.0, body_force=(1e-5, 0.0, 0.0), friction=0.05)
    o.fluid_init()
    o.step(STEPS)
    u = o.velocity()
    assert np.abs(u[:, 0, :, 0] - u[:, 1, :, 1]).max() == 0.0
    return u[:, 0, :, 0]  # [3][ny]


@pytest.mark.parametrize("prec,scale,bound,drift_bound",
                         [("f32", 0, 1e-5, 1e-6), ("f16s", 12, 1e-3, 5e-6), ("bf16s", 12, 2e-2, 5e-5)])
def test_channel_profile_and_mass_drift_512x256x256(profile, prec, scale, bound, drift_bound):
    g = lbib.Sim(NX, NY, NZ, walls=True, tau=1.0, rho0=1.0, body_force=(1e-5, 0.0, 0.0), friction=0.05,
                 precision=prec, pop_scale_log2=scale)
    g.fluid_init()
    m0 = g.mass()
    g.step(STEPS)
    m1 = g.mass()
    u = g.velocity()
    g.close()
    num = 0.0
    den = 0.0
    for k in range(3):  # component by component to bound host memory
        d = u[k][:, 1:NY - 1, :].astype(np.float64) - profile[k][None, 1:NY - 1, None]
        num += float(np.sum(d * d))
        den += float(np.sum(profile[k][1:NY - 1] ** 2)) * NX * NZ
    err = (num / den) ** 0.5
    drift = abs(m1 - m0) / m0
    print(f"\n{prec}: relative L2 vs FP64 oracle {err:.3e}, mass drift {drift:.3e} over {STEPS} steps, "
          f"u_max {profile[0].max():.4e}")
    assert err <= bound, err
    assert drift <= drift_bound, drift
