"""The weight blobs the tests and the bench feed nis_load_weights follow the layout that
include/nis.h documents: header words, tensor order and sizes, checksum."""
import struct

import numpy as np

import synth


def _sizes_lattice():
    out = []
    for _ in range(12):
        out += [16 * 27, 16, 16 * 16 * 27, 16]                    # CNN w1, b1, w2, b2
    for _ in range(12):
        out += [2 * 8, 2, 3 * 2, 3]                                # SE
    for d in (225, 225, 80):
        for _ in range(12):
            out += [200 * (d + 5), 200, 200 * 200, 200]            # blocks
    for _ in range(3):
        out += [200 * 400, 200]                                    # merges
    out += [200 * 600, 200, 200 * 200, 200, 3 * 200, 3]            # head
    return out


def _sizes_paper():
    counts = (6, 8, 12, 16, 24, 32, 48, 48, 32, 16, 16, 8)
    out = [11, 1]                                                  # level weights, bias
    for _ in range(12):
        out += [2 * 8, 2, 3 * 2, 3]
    for _ in range(3):
        for n in counts:
            out += [200 * (n + 5), 200, 200 * 200, 200]
    for _ in range(3):
        out += [200 * 400, 200]
    out += [200 * 600, 200, 200 * 200, 200, 3 * 200, 3]
    return out


def _check(blob, tensors, sizes, header):
    words = struct.unpack("<16I", blob[:64])
    n_floats, checksum = struct.unpack("<QQ", blob[64:80])
    for i, v in header.items():
        assert words[i] == v, (i, words[i], v)
    assert [t.size for t in tensors] == sizes
    assert n_floats == sum(sizes) and len(blob) == 80 + 4 * n_floats
    payload = np.frombuffer(blob[80:], dtype="<u4").astype(np.uint64)
    weights = 2 * np.arange(payload.size, dtype=np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        assert int(np.sum(payload * weights, dtype=np.uint64)) == checksum
    # the payload is the tensors in order
    flat = np.concatenate([np.ascontiguousarray(t, dtype="<f4").ravel() for t in tensors])
    np.testing.assert_array_equal(np.frombuffer(blob[80:], dtype="<f4"), flat)


def test_lattice_blob_layout():
    w = synth.make_weights(3, 8.0)
    _check(synth.pack_weights(w), synth.weight_tensors(w), _sizes_lattice(),
           {0: 0x5753494E, 1: 1, 2: 0, 3: 80, 4: 12, 5: 8, 6: 225, 7: 16, 8: 2, 9: 200, 10: 5,
            11: 3, 12: 80})


def test_paper_blob_layout():
    w = synth.make_weights_paper(3, 8.0)
    _check(synth.pack_weights_paper(w), synth.weight_tensors_paper(w), _sizes_paper(),
           {0: 0x5753494E, 1: 1, 2: 1, 3: 80, 4: 12, 5: 8, 6: 266, 7: 0, 8: 2, 9: 200, 10: 5,
            11: 3, 12: 11})
    lw = w["level"]["w"]
    assert lw.shape == (11,) and np.all(lw > 0) and 0.5 < lw.sum() < 1.5
