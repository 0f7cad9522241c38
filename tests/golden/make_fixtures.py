"""Writes tests/golden/modexp_small.txt: a few constant-time exponentiations and Montgomery
products (Alg. 5-7) computed by the CPU oracle on seeded inputs, as hex text. The paper prints
no worked numeric example, so the stored values come from the oracle (this script calls only
oracle/ and the seeded generator); tests check them against Python's own integers too.

    python tests/golden/make_fixtures.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def main():
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    import seeded_inputs as si
    lines = ["# bits window N a e modexp(a,e,N) mont(a,a,N)   (hex, one instance per line)"]
    for bits in (256, 1024, 2048):
        b = si.make_batch(0, "test", 3, bits, sub=9100 + bits)
        a = b.a.copy()
        e = b.e.copy()
        a[1] = b.N[1] - np.array([1] + [0] * (b.n - 1), np.uint32)      # N - 1
        e[2, :] = 0xFFFFFFFF                                              # all-ones exponent
        y = oracle.modexp(a, e, bits, b.N)
        m = oracle.mont_def(a, a, b.N)
        for k in range(3):
            lines.append(" ".join([str(bits), "5"] + [hex(si.to_int(v)) for v in (b.N[k], a[k], e[k], y[k], m[k])]))
    with open(os.path.join(HERE, "modexp_small.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
