"""Write tests/golden/oracle_digests.json: SHA-256 digests of the oracle's outputs
on seeded synthetic inputs. Calls only the oracle (and the input generator).

The digests pin the oracle and the generator across hosts (x86_64 and aarch64,
different compilers): a run elsewhere that disagrees has drifted, e.g. through
floating-point contraction in the float32 variant.

usage: python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1710_07745_gb300 import synth  # noqa: E402


def digest(a) -> str:
    return hashlib.sha256(a.tobytes()).hexdigest()


def cases():
    small = synth.small()
    yield "synth_small", small
    yield "canny_u8_small", oracle.canny_u8(small)
    yield "classify_u8_small", oracle.classify_u8(small)
    e, M, cls = oracle.canny_f32(small, want_stages=True)
    yield "canny_f32_small", e
    yield "magnitude_f32_small", M
    odd = synth.image(77, 333, 97, 6, 6, 12)
    yield "synth_333x97", odd
    yield "canny_u8_333x97", oracle.canny_u8(odd)


def main():
    out = {name: digest(a) for name, a in cases()}
    with open(os.path.join(HERE, "oracle_digests.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
