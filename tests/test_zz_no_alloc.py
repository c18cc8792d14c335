"""The allocation-free neighbour-list entry point, for callers that may not allocate device memory.

fnn_build_neighbors_static keeps all of its scratch in an array compiled into the library, so it can
serve code that owns every device buffer itself (a framework's memory pool) or that must not pay
for cudaMalloc's device-wide synchronisation.  The test allocates the outputs (the entry point does
not), calls it through the C ABI twice in a row on different systems, and requires each list to be
identical to the one the allocating entry point builds (lists are compared bit-exactly, as in every
neighbour-list test here).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from conftest import structure

pytestmark = pytest.mark.gpu


def _static_list(fnn, ds, R, cap):
    import torch
    row_ptr = torch.zeros(ds.n_atoms + 1, dtype=torch.int32, device="cuda")
    nbr = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda")
    shift4 = torch.zeros((max(cap, 1), 4), dtype=torch.int8, device="cuda")
    nnz = ctypes.c_int64(-1)
    cs = ds.c()
    code = fnn.lib.fnn_build_neighbors_static(ctypes.byref(cs), R, row_ptr.data_ptr(), nbr.data_ptr(),
                                              shift4.data_ptr(), cap, ctypes.byref(nnz),
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, nnz.value, row_ptr.cpu().numpy(), nbr.cpu().numpy()[:nnz.value], shift4.cpu().numpy()[:nnz.value, :3]


def _reference_list(fnn, ds, skin):
    ctx = fnn.Context(1, skin=skin)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    return fnn.nlist_export(nl, ds.n_atoms)


def test_static_entry_point_matches_allocating_one_twice_in_a_row():
    from paper_2405_01491_b300 import fnn
    # a periodic box with a skin, then a ragged gas-phase batch: the second call must not see the first's data;
    # then a dense box at R = 6.5 A whose rows hold about 158 entries (beyond the 128 that are sorted by
    # element: such rows keep the traversal order, on both entry points)
    for name, skin in (("box1500", 1.0), ("batch64", 0.0), ("box1100", 1.4)):
        ds = fnn.DeviceSystem.from_structures(structure(name))
        R = 5.1 + skin
        row_ref, nbr_ref, sh_ref = _reference_list(fnn, ds, skin)
        code, nnz, row_ptr, nbr, sh = _static_list(fnn, ds, R, cap=len(nbr_ref) + 64)
        assert code == 0, code
        assert nnz == len(nbr_ref)
        assert np.array_equal(row_ptr, row_ref)
        assert np.array_equal(nbr, nbr_ref)
        assert np.array_equal(sh, sh_ref)
        if name == "box1100":
            assert np.diff(row_ptr).max() > 128


def test_static_entry_point_limits():
    from paper_2405_01491_b300 import fnn, synth
    s = structure("box1500")
    ds = fnn.DeviceSystem.from_structures(s)
    # list larger than the caller's buffers: the size needed comes back, nothing beyond cap is written
    code, nnz, *_ = _static_list(fnn, ds, 5.1, cap=1000)
    assert code == -4 and nnz > 1000
    # more atoms than the static scratch holds: rejected before any GPU work
    big = synth.mix_box(9000, (9000 / 0.1) ** (1 / 3), seed=5)
    code, nnz, *_ = _static_list(fnn, fnn.DeviceSystem.from_structures(big), 5.1, cap=10)
    assert code == -4 and nnz == 0


def test_static_entry_point_rejects_overlapping_offsets():
    from paper_2405_01491_b300 import fnn, synth
    s = structure("box300")
    N = s.n_atoms
    # consistent structure by structure, but [0, N) twice: every structure is dropped, nothing is listed
    over = synth.Structures(s.Z, s.pos, np.array([0, N, 0, N], np.int32), np.repeat(s.cell, 3, 0),
                            np.repeat(s.pbc, 3))
    code, nnz, row_ptr, *_ = _static_list(fnn, fnn.DeviceSystem.from_structures(over), 5.1, cap=1000)
    assert code == -1 and nnz == 0 and not row_ptr.any()
    # and the next call on the shared scratch is clean again
    ds = fnn.DeviceSystem.from_structures(s)
    row_ref, nbr_ref, _ = _reference_list(fnn, ds, 0.0)
    code, nnz, row_ptr, nbr, _ = _static_list(fnn, ds, 5.1, cap=len(nbr_ref))
    assert code == 0 and np.array_equal(row_ptr, row_ref) and np.array_equal(nbr, nbr_ref)
