"""Lanczos checkpoint files (host logic, no GPU): round trip, and every kind
of damage -- a flipped byte, a truncated file, a missing array, inconsistent
shapes -- raises CheckpointError (the library's own check of the state runs
in tests/test_gpu_checkpoint.py)."""
import numpy as np
import pytest

from paper_1408_3036_gb300.checkpoint import CheckpointError, load_lanczos, save_lanczos


def _state(k=6, n=64, seed=0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return Q.T.copy(), rng.standard_normal(k), rng.uniform(0.5, 1.0, k - 1)


def test_round_trip(tmp_path):
    Q, a, b = _state()
    p = tmp_path / "ck.npz"
    save_lanczos(p, Q, a, b, 0.25)
    Q2, a2, b2, om = load_lanczos(p)
    assert np.array_equal(Q, Q2) and np.array_equal(a, a2) and np.array_equal(b, b2) and om == 0.25


def test_flipped_byte_is_detected(tmp_path):
    Q, a, b = _state()
    p = tmp_path / "ck.npz"
    save_lanczos(p, Q, a, b, 0.0)
    raw = bytearray(p.read_bytes())
    # flip one byte inside the stored Q (the first array's data, past the headers)
    raw[len(raw) // 3] ^= 0x40
    p.write_bytes(bytes(raw))
    with pytest.raises(CheckpointError):
        load_lanczos(p)


def test_truncated_file_is_detected(tmp_path):
    Q, a, b = _state()
    p = tmp_path / "ck.npz"
    save_lanczos(p, Q, a, b, 0.0)
    raw = p.read_bytes()
    p.write_bytes(raw[: len(raw) // 2])
    with pytest.raises(CheckpointError):
        load_lanczos(p)


def test_missing_array_and_bad_shapes(tmp_path):
    Q, a, b = _state()
    p = tmp_path / "ck.npz"
    np.savez(p, Q=Q, alpha=a, omega=np.float64(0.0), sha256=np.array("0"))
    with pytest.raises(CheckpointError):
        load_lanczos(p)
    np.savez(p, Q=Q, alpha=a[:-1], beta=b, omega=np.float64(0.0), sha256=np.array("0"))
    with pytest.raises(CheckpointError):
        load_lanczos(p)


def test_a_changed_value_with_a_stale_digest(tmp_path):
    Q, a, b = _state()
    p = tmp_path / "ck.npz"
    save_lanczos(p, Q, a, b, 0.0)
    with np.load(p) as f:
        d = {k: f[k] for k in f.files}
    d["beta"] = d["beta"].copy()
    d["beta"][1] *= 1.0 + 1e-15
    np.savez(p, **d)
    with pytest.raises(CheckpointError):
        load_lanczos(p)
