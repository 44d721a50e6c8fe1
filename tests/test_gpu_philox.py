"""The step's random-number generator on the device (qed_philox_blocks, both forms of the
key schedule): the published Philox4x32-10 known-answer vectors, and cuRAND's own
Philox4x32-10 device function on the same (counter, key) for many random counters,
including the all-ones words whose key and counter arithmetic wraps."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    return torch.device("cuda")


def _run(ctr_np, key):
    ctr = torch.from_numpy(ctr_np.astype(np.uint32).view(np.int32)).cuda()
    out = torch.empty((ctr.shape[0], 8), dtype=torch.int32, device="cuda")
    q.qed_philox_blocks(ctr, key, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def _kat():
    rows = []
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([int(w, 16) for w in line.split()])
    return rows


def test_known_answer_vectors(dev):
    for v in _kat():
        got = _run(np.array([v[0:4]]), v[4] | (v[5] << 32))[0]
        assert list(got[0:4]) == v[6:10]
        assert list(got[4:8]) == v[6:10]


@pytest.fixture(scope="module")
def curand_ref(dev, tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    so = str(tmp_path_factory.mktemp("curand") / "libcurand_philox_ref.so")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                        "-o", so, os.path.join(HERE, "curand_philox_ref.cu")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = C.CDLL(so)
    L.curand_philox_ref.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint64]
    L.curand_philox_ref.restype = C.c_int
    return L


@pytest.mark.parametrize("key", [0, 0xFFFFFFFFFFFFFFFF, 0x243F6A8885A308D3, 20240917])
def test_matches_curand(dev, curand_ref, key):
    rng = np.random.default_rng(key & 0xFFFF)
    n = 100_003
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:64] = 0xFFFFFFFF                      # carries in every word
    ctr[64:128, 2] = np.arange(64)             # the step's counters: (id lo, id hi, step, draw)
    ctr[64:128, 3] = np.arange(64) % 4
    got = _run(ctr, key)
    c = torch.from_numpy(ctr.view(np.int32)).cuda()
    ref = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    assert curand_ref.curand_philox_ref(c.data_ptr(), key, ref.data_ptr(), n) == 0
    ref = ref.cpu().numpy().view(np.uint32)
    assert np.array_equal(got[:, 0:4], ref)
    assert np.array_equal(got[:, 4:8], ref)


def test_empty_and_validation(dev):
    z = torch.empty((0, 4), dtype=torch.int32, device="cuda")
    q.qed_philox_blocks(z, 1, torch.empty((0, 8), dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        q.qed_philox_blocks(torch.empty((3, 4), dtype=torch.int32, device="cuda"), 1,
                            torch.empty((3, 4), dtype=torch.int32, device="cuda"))
