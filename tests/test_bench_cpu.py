"""Host-side checks of the benchmark script that need no GPU."""
import os


def test_profile_commands_parse():
    """Every bench.py command line in the committed profile summaries is
    accepted by the benchmark's argument parser."""
    import glob
    import re
    import shlex
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    found = 0
    for path in glob.glob(os.path.join(root, "profiles", "*.md")):
        text = open(path).read().replace("\\\n", " ")
        for m in re.finditer(r"python bench\.py([^>&\n]*)", text):
            bench.build_parser().parse_args(shlex.split(m.group(1)))
            found += 1
    assert found >= 2
