"""The batched streaming passes map a tile to its ensemble with two warp ballots
(find_ens_warp: the offsets 32 apart, then the 32 from there) instead of a per-thread binary
search (find_ens).  Both must name the last ensemble whose first tile is at or below the
tile, for any table of up to 1024 ensembles, empty ensembles (repeated offsets) included."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    so = str(tmp_path_factory.mktemp("enslookup") / "libens_lookup_probe.so")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                        "-Xcompiler", "-fPIC", "-I", os.path.join(HERE, "..", "include"), "-o", so,
                        os.path.join(HERE, "ens_lookup_probe.cu")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = C.CDLL(so)
    L.ens_lookup_eval.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    L.ens_lookup_eval.restype = C.c_int

    def ev(off, g):
        od = torch.from_numpy(np.ascontiguousarray(off, np.uint32).view(np.int32)).cuda()
        gd = torch.from_numpy(np.ascontiguousarray(g, np.uint32).view(np.int32)).cuda()
        wa = torch.empty(len(g), dtype=torch.int32, device="cuda")
        sa = torch.empty_like(wa)
        assert L.ens_lookup_eval(od.data_ptr(), len(off) - 1, gd.data_ptr(), len(g), wa.data_ptr(), sa.data_ptr()) == 0
        return wa.cpu().numpy(), sa.cpu().numpy()
    return ev


def _table(rng, n, p_empty):
    tiles = rng.integers(1, 40, n)
    tiles[rng.random(n) < p_empty] = 0     # empty ensembles: repeated offsets
    tiles[-1] = max(tiles[-1], 1)          # something to look up
    return np.concatenate([[0], np.cumsum(tiles)]).astype(np.uint32)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 63, 64, 65, 100, 511, 1000, 1023, 1024])
def test_ballot_lookup_equals_binary_search(probe, n):
    rng = np.random.default_rng(100 + n)
    for p_empty in (0.0, 0.3):
        off = _table(rng, n, p_empty)
        g = np.arange(off[-1], dtype=np.uint32)        # every tile
        w, s = probe(off, g)
        # the definition: the last e < n with off[e] <= g
        ref = np.searchsorted(off[:n], g, side="right") - 1
        assert np.array_equal(s, ref), n
        assert np.array_equal(w, ref), n
        # every answer is a non-empty ensemble that holds the tile
        assert np.all(off[w] <= g) and np.all(g < off[w + 1])
