"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/fnn.h declares
(no CUDA call is made: these run on a machine without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fnn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fnn_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2405_01491_b300 import build
    so = build.build()
    lib = ctypes.CDLL(so)
    names = declared_symbols()
    assert "fnn_energy_forces" in names and "fnn_build_neighbors" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_fills_defaults():
    from paper_2405_01491_b300 import fnn
    cfg = fnn.Config()
    fnn.lib.fnn_config_default(ctypes.byref(cfg))
    assert (cfg.rc_rad, cfg.rc_ang, cfg.eta_rad, cfg.eta_ang, cfg.zeta) == (5.1, 3.5, 19.7, 12.5, 14.1)
    assert cfg.n_members == 1 and cfg.skin == 0.0


def test_create_rejects_bad_config_without_device():
    from paper_2405_01491_b300 import fnn
    cfg = fnn.Config()
    fnn.lib.fnn_config_default(ctypes.byref(cfg))
    cfg.rc_ang = 6.0   # angular cutoff beyond the radial one
    h = ctypes.c_void_p()
    assert fnn.lib.fnn_create(ctypes.byref(h), ctypes.byref(cfg)) == -1
    cfg.rc_ang = 3.5
    cfg.n_members = 9
    assert fnn.lib.fnn_create(ctypes.byref(h), ctypes.byref(cfg)) == -1


def test_weight_file_format(tmp_path):
    import numpy as np
    from paper_2405_01491_b300 import fnn, synth
    w = synth.xavier_weights(1)
    p = tmp_path / "w.fnnw"
    fnn.save_weights(str(p), w)
    raw = p.read_bytes()
    assert raw[:4] == b"FNNW"
    assert np.frombuffer(raw[4:12], "<i4").tolist() == [1, 1]
    n = 8 + 4 + 4 * sum(getattr(w, k).size for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"))
    assert len(raw) == n
