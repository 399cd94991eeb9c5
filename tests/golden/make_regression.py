"""Writes regression_seed12345.txt from the oracle alone (no GPU code)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import oracle  # noqa: E402


def main():
    o = oracle()
    x, c = o.seeded_state(12345)
    out, _, _ = o.generate(x, c, 8)
    J = (1 << 120) + 12345
    xj, cj = o.jump(x, c, J)
    with open(os.path.join(HERE, "regression_seed12345.txt"), "w") as f:
        f.write("# Written by tests/golden/make_regression.py from the CPU oracle only.\n")
        f.write("# seed 12345: first 8 outputs of Algorithm 2; jump by 2^120 + 12345:\n")
        f.write("# sum of the 97 jumped words and the jumped c.\n")
        f.write(f"jump {J}\n")
        f.write(f"xsum {int(xj.astype(np.uint64).sum())}\n")
        f.write(f"cjump {cj}\n")
        for v in out:
            f.write(f"{int(v)}\n")


if __name__ == "__main__":
    main()
