"""Reader for the bracketed text fixtures in tests/golden/."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load_blocks(name):
    blocks, cur = {}, None
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                blocks[cur] = []
                continue
            blocks[cur].append([float(v) for v in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}
