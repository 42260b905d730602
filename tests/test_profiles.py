"""CPU checks of the committed ncu summaries under profiles/: short text files, each
giving the full ncu command that produced it (with --clock-control none) over committed
files only, and the traffic table that gates roofline.traffic has a row per timed family."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_profiles_are_short_text_with_their_command():
    files = sorted(os.listdir(PROFILES))
    assert files
    for fn in files:
        path = os.path.join(PROFILES, fn)
        assert fn.endswith((".md", ".txt")), fn
        text = open(path).read()
        assert len(text) < 16 * 1024, fn
        assert re.search(r"\bncu\b", text) and "--clock-control none" in text, fn
        assert "python bench.py" in text, fn        # the command runs the committed bench
        assert "_work" not in text, fn


def test_traffic_table_covers_the_timed_families():
    # one row per timed family: DRAM bytes per cell and the 16-hex-digit source digest that
    # bench.py compares before reporting roofline.traffic.  The bytes are at least the
    # algorithmic bytes less what the L2 (126 MB on a GB300) can still hold as dirty lines
    # when the kernel ends, per cell of the 384^3 capture.
    import bench
    rows = {}
    with open(os.path.join(PROFILES, "ncu_traffic.txt")) as fh:
        for line in fh:
            cols = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cols) >= 5 and cols[0] in ("down0", "up0", "df0"):
                rows[cols[0]] = (float(cols[3]), cols[4])
    assert set(rows) == {"down0", "up0", "df0"}
    for fam, (bpc, digest) in rows.items():
        assert bpc >= bench.BYTES_PER_CELL[fam] - 126e6 / 384**3, fam
        assert re.fullmatch(r"[0-9a-f]{16}", digest), fam
