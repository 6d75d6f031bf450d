"""The on-disk cache of generated graphs (no GPU): a cached graph equals a generated
one, other parameters get their own file, and a file whose header or checksum does not
match is regenerated instead of being used."""
import os

import numpy as np

import inputs


def _files(d):
    return sorted(f for f in os.listdir(d) if f.endswith(".csr"))


def test_cached_graph_equals_the_generated_one(tmp_path):
    d = str(tmp_path)
    rp0, col0 = inputs.rmat_csr(12, 8, 5)
    rp1, col1 = inputs.rmat_csr(12, 8, 5, cache_dir=d)   # generates and writes
    assert len(_files(d)) == 1
    rp2, col2 = inputs.rmat_csr(12, 8, 5, cache_dir=d)   # reads
    for rp, col in ((rp1, col1), (rp2, col2)):
        np.testing.assert_array_equal(rp, rp0)
        np.testing.assert_array_equal(col, col0)
        assert rp.dtype == np.int64 and col.dtype == np.int32
    inputs.rmat_csr(12, 8, 6, cache_dir=d)               # another seed: another file
    inputs.rmat_csr(12, 4, 5, cache_dir=d)               # another degree: another file
    assert len(_files(d)) == 3


def test_damaged_cache_files_are_regenerated(tmp_path):
    d = str(tmp_path)
    rp0, col0 = inputs.rmat_csr(11, 8, 7, cache_dir=d)
    path = os.path.join(d, _files(d)[0])
    size = os.path.getsize(path)
    # flip one byte of the column array: the checksum no longer matches
    with open(path, "r+b") as f:
        f.seek(size - 3)
        b = f.read(1)
        f.seek(size - 3)
        f.write(bytes([b[0] ^ 0xFF]))
    rp1, col1 = inputs.rmat_csr(11, 8, 7, cache_dir=d)
    np.testing.assert_array_equal(col1, col0)
    np.testing.assert_array_equal(rp1, rp0)
    # a truncated file, and a file that is not a cache file at all
    with open(path, "r+b") as f:
        f.truncate(size // 2)
    np.testing.assert_array_equal(inputs.rmat_csr(11, 8, 7, cache_dir=d)[1], col0)
    with open(path, "wb") as f:
        f.write(b"not a graph")
    np.testing.assert_array_equal(inputs.rmat_csr(11, 8, 7, cache_dir=d)[1], col0)
    assert os.path.getsize(path) == size  # rewritten whole


def test_cache_directory_from_the_environment(tmp_path, monkeypatch):
    monkeypatch.setenv("FORA_GRAPH_CACHE", str(tmp_path))
    rp, col = inputs.rmat_csr(10, 4, 3)
    assert len(_files(str(tmp_path))) == 1
    monkeypatch.delenv("FORA_GRAPH_CACHE")
    rp2, col2 = inputs.rmat_csr(10, 4, 3)
    np.testing.assert_array_equal(col2, col)
