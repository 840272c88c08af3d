"""vsie_load rejects missing, foreign and truncated files before touching the
GPU (host-side checks of the operator file header)."""
import pytest


def test_load_rejects_bad_files(tmp_path):
    from paper_2206_12409_gb300 import vsie as V
    with pytest.raises(V.VsieError):
        V.vsie_load(tmp_path / "missing.vsie")
    bad = tmp_path / "bad.vsie"
    bad.write_bytes(b"NOTVSIE!" + b"\0" * 64)
    with pytest.raises(V.VsieError):
        V.vsie_load(bad)
    trunc = tmp_path / "trunc.vsie"
    trunc.write_bytes(b"VSIEOPS1" + (1).to_bytes(4, "little") + b"\0" * 10)
    with pytest.raises(V.VsieError):
        V.vsie_load(trunc)
