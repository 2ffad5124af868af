"""Host-side checks of the checkpoint reader (no GPU): files that lack a field or carry another
format version are refused before any handle is created."""
import numpy as np
import pytest

from paper_2007_06427_gb300 import checkpoint as C


def _fields(**over):
    f = dict(L=22.0, nx=32, ns=np.array([32], dtype=np.int64), mode=0, scheme=1, dtau=0.15,
             tol=1e-10, switch_tol=0.0, band=np.zeros(2 * 11 * 21), T=np.array([40.0]),
             prec=np.zeros(1, dtype=np.int32), steps=np.zeros(1, dtype=np.int64),
             status=np.zeros(1, dtype=np.int32), version=C.VERSION)
    f.update(over)
    return f


@pytest.mark.parametrize("drop", ["band", "T", "version", "ns", "status"])
def test_missing_field_is_refused(tmp_path, drop):
    f = _fields()
    del f[drop]
    path = tmp_path / "ck.npz"
    np.savez(path, **f)
    with pytest.raises(ValueError, match=drop):
        C.resume(str(path))


def test_other_version_is_refused(tmp_path):
    path = tmp_path / "ck.npz"
    np.savez(path, **_fields(version=C.VERSION + 1))
    with pytest.raises(ValueError, match="version"):
        C.resume(str(path))
