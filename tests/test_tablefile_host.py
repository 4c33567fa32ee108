"""Host-side validation of the paper's table files (section 2): malformed files are
refused before any device work (no GPU needed)."""
import struct

import oracle as O


def _cb():
    import paper_1601_00636_gb300 as cb
    return cb


def _files(tmp_path, blob, recs):
    b, p = tmp_path / "b.bin", tmp_path / "p.bin"
    b.write_bytes(blob)
    p.write_bytes(recs)
    return str(b), str(p)


def test_malformed_files_are_refused(tmp_path):
    cb = _cb()
    blob, recs = O.paper_table_files([11, 13])
    cases = [
        (blob, recs[:-1], cb.EINVAL),                                         # partial record
        (blob, b"", cb.EINVAL),                                               # no record
        (blob[:-1], recs, cb.ERANGE),                                         # table past the end
        (blob, recs[:8] + struct.pack("<hxxI", 15, 16), cb.EINVAL),           # 15 is not prime
        (blob, recs[:8] + struct.pack("<hxxI", 13, 10 ** 6), cb.ERANGE),      # offset past the end
        (blob, recs[:8] + struct.pack("<hxxI", -3, 16), cb.EINVAL),           # negative short
    ]
    padded = bytearray(blob)
    padded[15] |= 0x80                                                        # pad bit of u_11 (121 bits)
    cases.append((bytes(padded), recs, cb.EINVAL))
    for blob_i, recs_i, code in cases:
        st, h = cb.cuboid_tables_import_status(*_files(tmp_path, blob_i, recs_i))
        assert st == code and h is None
    st, _ = cb.cuboid_tables_import_status(str(tmp_path / "missing.bin"), str(tmp_path / "p.bin"))
    assert st == cb.EINVAL
    st, _ = cb.cuboid_tables_import_status(*_files(tmp_path, blob, recs), flags=cb.BUILD_FULL)
    assert st == cb.EINVAL
