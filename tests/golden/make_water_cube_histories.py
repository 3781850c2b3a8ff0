"""Write tests/golden/water_cube_histories.txt: per-history step and
secondary counts and deposited energy of the first 200 primaries of the
photon-only water cube, from the CPU oracle only (a regression record of the
oracle; the GPU parity tests compare with the oracle run live)."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2503_17608_gb300 import workloads as wl  # noqa: E402

N = 200


def histories():
    prob = wl.water_cube_problem()
    prim = wl.water_cube_primaries(N)
    hist, edep = oracle.World(prob).run(prim, n_threads=1)
    return hist, edep


def main():
    hist, edep = histories()
    path = os.path.join(HERE, "water_cube_histories.txt")
    with open(path, "w") as f:
        f.write("# photon-only water cube, 10 MeV photons from the origin along +z, seed 20250321, first "
                f"{N} primaries\n")
        f.write("# written by tests/golden/make_water_cube_histories.py from the CPU oracle\n")
        f.write("# primary steps secondaries edep_MeV escaped_MeV\n")
        for i in range(N):
            f.write(f"{i} {int(hist['steps'][i])} {int(hist['secondaries'][i])} {edep[i].sum():.17g} "
                    f"{hist['escaped'][i]:.17g}\n")
    print(path)


if __name__ == "__main__":
    main()
