"""Write the Lorenz-Mie reference intensities of the bench workloads.

Calls only oracle/ (the Lorenz-Mie series of oracle/mie.py); the output text
files are data read by bench.py and the tests:
  mie_sphere_x5_m1.33.txt      3D sphere (Sec. 3.4 geometry), x = 5, n = 1.33,
                               theta = 0..180 deg by 1 deg, phi = 0, 45, 90 deg
  mie_cylinder_x5_m1.5.txt     2D cylinder (Sec. 3.2 geometry), x = 5, n = 1.5,
                               TM (E along the axis) and TE, theta = 0..180 deg
  mie_batch_cylinders_seed20251011.txt
                               TM intensity of each of the 32 seeded cylinders of the
                               batched workload (workloads.batched_problems: the
                               seeded x and n = sqrt(eps_r) of every problem),
                               theta = 0..180 deg
Run:  python tests/golden/make_mie_reference.py
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mie  # noqa: E402
import workloads as W  # noqa: E402  (seeded sizes only: no lattice arithmetic)


def main():
    th = np.radians(np.arange(181.0))
    cols = [np.arange(181.0)]
    for ph in (0.0, 45.0, 90.0):
        cols.append(mie.sphere_intensity(th, np.full(181, math.radians(ph)), 5.0, 1.33))
    np.savetxt(os.path.join(HERE, "mie_sphere_x5_m1.33.txt"), np.stack(cols, 1),
               header="Lorenz-Mie |S|^2 of a sphere, x = 5, m = 1.33 (oracle/mie.py)\n"
                      "theta_deg  phi=0  phi=45  phi=90", fmt="%.12e")
    cols = [np.arange(181.0), mie.cylinder_intensity(th, 5.0, 1.5, "TM"),
            mie.cylinder_intensity(th, 5.0, 1.5, "TE")]
    np.savetxt(os.path.join(HERE, "mie_cylinder_x5_m1.5.txt"), np.stack(cols, 1),
               header="Lorenz-Mie |S|^2 of an infinite cylinder, x = 5, m = 1.5 (oracle/mie.py)\n"
                      "theta_deg  TM(E_along_axis)  TE(H_along_axis)", fmt="%.12e")
    probs = W.batched_problems(32, 20251011)
    cols = [np.arange(181.0)]
    desc = []
    for p in probs:
        x, m = p.meta["x"], p.meta["m"]
        cols.append(mie.cylinder_intensity(th, x, m, "TM"))
        desc.append(f"n={p.shape[0]} x={x:.10g} m={m:.10g} lambda={p.wave.wavelength:g}")
    np.savetxt(os.path.join(HERE, "mie_batch_cylinders_seed20251011.txt"), np.stack(cols, 1),
               header="Lorenz-Mie TM |S|^2 of the 32 cylinders of workloads.batched_problems(32, 20251011) "
                      "(oracle/mie.py)\ncolumns: theta_deg, then one per problem in order:\n" + "\n".join(desc),
               fmt="%.12e")


if __name__ == "__main__":
    main()
