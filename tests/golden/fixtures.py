"""Readers for the hand-derived text fixtures in this folder."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load_stream_fixture(name):
    m = eb_log2 = None
    amps = {}
    hexparts = []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *rest = line.split()
            if key == "m":
                m = int(rest[0])
            elif key == "eb_log2":
                eb_log2 = int(rest[0])
            elif key == "amp":
                amps[int(rest[0])] = (float(rest[1]), float(rest[2]))
            elif key == "hex":
                hexparts.extend(rest)
    block = np.zeros(2 << m, dtype=np.float32)
    for i, (re, im) in amps.items():
        block[2 * i] = re
        block[2 * i + 1] = im
    stream = bytes.fromhex("".join(hexparts))
    return m, 2.0 ** eb_log2, block, stream


def load_ties():
    e = None
    rows = []
    with open(os.path.join(HERE, "quantize_ties.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            a, b = line.split()
            if a == "e":
                e = int(b)
            else:
                rows.append((float(a), int(b)))
    return e, rows
