"""Reader for the small text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_cases(name: str = "objective_hand.txt"):
    """Parse `case <id>` blocks of `key values...` lines (comments start with #)."""
    cases = {}
    cur = None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "case":
                cur = {}
                cases[vals[0]] = cur
                continue
            nums = [float(v) for v in vals]
            if key == "shape":
                cur["shape"] = tuple(int(v) for v in nums)          # nz ny nx
            elif key == "psf":
                px, py, pz = (int(v) for v in nums[:3])
                nz = cur["shape"][0]
                taps = np.array(nums[3:], np.float32).reshape(pz, py, px)
                cur["psf"] = np.broadcast_to(taps, (nz, pz, py, px)).copy()
            elif key == "params":
                lam, delta, eta, xmin, xmax = nums
                cur["params"] = dict(lam=lam, delta=delta, eta=eta, xmin=xmin, xmax=xmax)
            elif key == "penalty":                                   # mode, kappa
                cur["params"].update(penalty=int(nums[0]), kappa=nums[1])
            elif key in ("y", "x", "Hx", "grad"):
                cur[key] = np.array(nums).reshape(cur["shape"])
            else:
                cur[key] = nums[0] if len(nums) == 1 else np.array(nums)
    return cases
