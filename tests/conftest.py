import functools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@functools.lru_cache(maxsize=None)
def weights(n_members: int, seed: int = 0):
    from paper_2405_01491_b300 import synth
    return synth.xavier_weights(n_members, seed)


@functools.lru_cache(maxsize=None)
def structure(name: str):
    from paper_2405_01491_b300 import synth
    return {
        "gas24": synth.gas24,
        "water216": synth.water216,
        "mix23558": synth.mix23558,
        "batch64": lambda: synth.ragged_batch(64, seed=40),
        "batch4096": synth.ragged_batch,
        "box300": lambda: synth.mix_box(300, (300 / 0.1) ** (1 / 3), seed=31),
        "box1500": lambda: synth.mix_box(1500, (1500 / 0.1) ** (1 / 3), seed=32,
                                         fractions=synth.MIX7),
        # a 20 A periodic box (3 cells per axis: every cell's stencil is the whole box, 1100 candidates,
        # more than the pair search stages in shared memory, so its per-centre traversal runs)
        "box1100": lambda: synth.mix_box(1100, 20.0, seed=36, fractions=synth.MIX7),
        # three periodic boxes in one batch: structures large enough that each one's float64 energy is
        # summed in several slices, with more than one such structure at once
        "boxes3": lambda: synth.concat([synth.mix_box(n, (n / 0.1) ** (1 / 3), seed=33 + k, fractions=synth.MIX7)
                                        for k, n in enumerate((700, 2600, 1500))], "boxes3"),
    }[name]()


@pytest.fixture
def W1():
    return weights(1)


@pytest.fixture
def W2():
    return weights(2)
