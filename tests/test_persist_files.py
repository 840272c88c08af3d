"""vsie_load rejects missing, foreign, truncated and inconsistent files before
touching the GPU (host-side checks of the operator file)."""
import ctypes as C
import struct

import numpy as np
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
    trunc.write_bytes(b"VSIEOPS1" + (3).to_bytes(4, "little") + b"\0" * 10)
    with pytest.raises(V.VsieError):
        V.vsie_load(trunc)


def _arr(a, fmt):
    a = np.asarray(a)
    return struct.pack("<q", a.size) + a.astype(fmt).tobytes()


def _operator_file(port_row, port_len):
    """A complete version-3 operator file: 2^3 vacuum body, one far RWG (a 1 x 1
    Z_ff, no ACA factors, no tensor trains), no near RWG, and a port table."""
    from paper_2206_12409_gb300 import vsie as V
    g = V.make_grid((2, 2, 2), 1e-3, (0.0, 0.0, 0.0))
    o = V.make_options()
    nb = 8
    out = b"VSIEOPS1" + struct.pack("<I", 3) + bytes(g) + struct.pack("<d", 298e6) + bytes(o)
    out += _arr(np.ones(nb), "<f8") + _arr(np.zeros(nb), "<f8")
    out += struct.pack("<iii", 1, 0, 3)                       # m_f, m_n, stencil
    out += _arr(np.array([1.0, 0.5]), "<f8")                  # Z_ff (1 x 1, re/im)
    out += struct.pack("<i", 0)                               # ACA rank
    out += bytes((C.c_int32 * 9)())                           # TT ranks (none)
    out += _arr(np.asarray(port_row, np.int64), "<i8") + _arr(np.asarray(port_len), "<f8")
    return out


@pytest.mark.parametrize("row,length", [(1, 0.01), (-1, 0.01), (0, float("nan")), (0, 0.0)])
def test_load_rejects_bad_port_table(tmp_path, row, length):
    """A port must name a surface unknown (row in [0, m_f + m_n)) and carry a
    finite positive edge length; otherwise vsie_rhs_ports would write outside
    the right-hand side.  The file is rejected with VSIE_EINVAL on the host."""
    from paper_2206_12409_gb300 import vsie as V
    f = tmp_path / "ports.vsie"
    f.write_bytes(_operator_file([row], [length]))
    with pytest.raises(V.VsieError) as e:
        V.vsie_load(f)
    assert e.value.status == V.VSIE_EINVAL
    assert "port" in str(e.value)


def test_valid_port_table_passes_the_file_checks(tmp_path):
    """Control for the test above: the same file with a valid port gets past
    every file check (without a GPU the context creation itself then fails)."""
    from paper_2206_12409_gb300 import vsie as V
    f = tmp_path / "ok.vsie"
    f.write_bytes(_operator_file([0], [0.01]))
    try:
        ctx = V.vsie_load(f)
    except V.VsieError as e:
        assert "operator file" not in str(e) and "port" not in str(e), str(e)
    else:
        V.vsie_destroy(ctx)
