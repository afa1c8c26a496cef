"""Checkpoint and resume (cem_save / cem_load): a context loaded from a
checkpoint continues bit for bit as the saved one does; files of another mesh,
truncated or corrupted files are rejected and leave the context as it was."""
import numpy as np
import pytest

from cem_inputs import hex_block, kuhn_block, plate_small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


def _state(sim):
    return [sim.field(f) for f in ("u", "v", "a", "X")], sim.crack_state(), sim.energy(), sim.info()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_is_bit_identical_through_crack_growth(CEM, precision, tmp_path):
    w = kuhn_block(13, 6, 3, 0.065, 0.03, 0.015, notch_length=0.03, jitter=0.15, E_cov=0.1, Gc_cov=0.2,
                   seed=3, traction=2e6)
    path = str(tmp_path / "ck.bin")
    a = CEM.from_workload(w, precision=precision)
    a.step(100)                     # the crack grows from about step 50 to step 300
    n_before = len(a.crack_state())
    a.save(path)
    a.step(300)
    b = CEM.from_workload(w, precision=precision)
    b.load(path)
    assert b.energy()["step"] == 100
    b.step(300)
    fa, ca, ea, ia = _state(a)
    fb, cb, eb, ib = _state(b)
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)
    assert ca == cb and ea == eb and ia == ib
    assert len(ca) > n_before > len(w.notch_tet)


def test_resume_hexahedra(CEM, tmp_path):
    w = hex_block(6, 4, 2, 0.03, 0.02, 0.01, jitter=0.1, seed=2, traction=1e6)
    path = str(tmp_path / "hex.bin")
    a = CEM.from_hex_workload(w)
    a.step(100)
    a.save(path)
    a.step(100)
    b = CEM.from_hex_workload(w)
    b.load(path)
    b.step(100)
    assert np.array_equal(a.field("u"), b.field("u")) and a.energy() == b.energy()


def test_load_rejects_other_meshes_and_bad_files(CEM, tmp_path):
    from paper_2508_04076_gb300 import CEMError
    path = str(tmp_path / "ck.bin")
    a = CEM.from_workload(plate_small())
    a.step(10)
    a.save(path)
    other = CEM.from_workload(kuhn_block(10, 4, 1, 0.05, 0.02, 0.005, notch_length=0.025))
    with pytest.raises(CEMError):
        other.load(path)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a checkpoint at all")
    with pytest.raises(CEMError):
        a.load(str(bad))
    trunc = tmp_path / "trunc.bin"
    trunc.write_bytes(open(path, "rb").read()[:300])
    b = CEM.from_workload(plate_small())
    with pytest.raises(CEMError):
        b.load(str(trunc))
    # a flipped bit inside an array: rejected by the file hash, the context left as it was
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0x40
    flip = tmp_path / "flip.bin"
    flip.write_bytes(bytes(raw))
    c = CEM.from_workload(plate_small())
    c.step(5)
    u5 = c.field("u")
    with pytest.raises(CEMError):
        c.load(str(flip))
    assert np.array_equal(c.field("u"), u5) and c.energy()["step"] == 5
    c.step(5)
    assert np.array_equal(c.field("u"), a.field("u")) and c.energy() == a.energy()


def test_load_rejects_indices_out_of_range(CEM, tmp_path):
    """A file with a valid hash whose element holds a node index past the node
    count (a file cem_save did not write) is rejected before anything reaches the
    device, and the context continues as it was."""
    from ckpt_reader import chunks, read, rehash
    from paper_2508_04076_gb300 import CEMError
    path = str(tmp_path / "ck.bin")
    a = CEM.from_workload(plate_small())
    a.step(10)
    a.save(path)
    H, _ = read(path)
    raw = bytearray(open(path, "rb").read())
    conn0 = chunks(raw)[19]            # X, u, v, a, f_ext (3 rows each), mass, 1/m, incidence offset and count
    assert conn0[1] == 4 * H["T"]
    for bad_value in (H["N"] + 5, -1):
        mod = bytearray(raw)
        mod[conn0[0]:conn0[0] + 4] = int(bad_value).to_bytes(4, "little", signed=True)
        bad = tmp_path / "bad.bin"
        bad.write_bytes(bytes(rehash(mod)))
        c = CEM.from_workload(plate_small())
        c.step(5)
        u5 = c.field("u")
        with pytest.raises(CEMError):
            c.load(str(bad))
        assert np.array_equal(c.field("u"), u5) and c.energy()["step"] == 5
        c.step(5)
        assert np.array_equal(c.field("u"), a.field("u")) and c.energy() == a.energy()
    # the same file with its hash recomputed but no index changed loads
    ok = tmp_path / "ok.bin"
    ok.write_bytes(bytes(rehash(raw)))
    d = CEM.from_workload(plate_small())
    d.load(str(ok))
    assert np.array_equal(d.field("u"), a.field("u"))
