"""Host-side parts of the region search (no GPU): the segment bound of Eq. 1.2 used by
the library, and the section 5 report file."""
import re

import oracle as O


def _cb():
    import paper_1601_00636_gb300 as cb
    return cb


def test_region_qmin_matches_oracle():
    cb = _cb()
    for p in list(range(1, 3000)) + [154000, 112618, 10 ** 6, 72796055]:
        assert cb.cuboid_region_qmin(p) == O.region_q_bounds(p)[0]


def test_region_qmin_past_p_max():
    """Rows the 64-bit region scan visits: p_max + 1 up to 2^32 - 1, including the values
    where ceil((p / 9)^(1/3)) steps (9 q^3 = p and its neighbours)."""
    cb = _cb()
    ps = [72796056, 72796057, 10 ** 8, 2 ** 31, 2 ** 32 - 2, 2 ** 32 - 1]
    for q in (200, 201, 500, 777, 780, 781):
        ps += [9 * q ** 3 - 1, 9 * q ** 3, 9 * q ** 3 + 1]
    for p in ps:
        if p < 2 ** 32:
            assert cb.cuboid_region_qmin(p) == O.region_q_bounds(p)[0], p


def test_report_file_format(tmp_path):
    """Section 5's report: a time stamp line, then the exit values of p, q and r_max."""
    cb = _cb()
    f = tmp_path / "report.txt"
    rep = {"p": 112618, "q": 5691455, "r_max": 131, "depth": 27, "pairs": 0, "n_surv": 0, "n_roots": 0}
    cb.cuboid_search_report_write(rep, str(f))
    cb.cuboid_search_report_write(dict(rep, p=112700, q=1), str(f))
    lines = f.read_text().splitlines()
    assert len(lines) == 4
    assert re.fullmatch(r"\d{4}-\d{1,2}-\d{1,2} \d\d:\d\d", lines[0])
    assert lines[1] == "Stop with p=112618, q=5691455, r_max=131"
    assert lines[3] == "Stop with p=112700, q=1, r_max=131"
