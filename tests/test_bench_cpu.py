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


def test_stored_oracle_images_are_of_the_benchmark_scans():
    """The oracle's stored MAP images (tests/golden) are of exactly the two
    scans the benchmark reconstructs per step (input digests) and of its
    shared prior scale (sigma_x from the first scan's weights), so the bench
    line's NRMSE compares like with like."""
    import hashlib
    import os
    import numpy as np
    import bench
    import synth
    y, lam = bench.make_inputs(2, 0)
    sx = synth.prior_sigma_x(lam[0], bench.WORKLOAD["n_views"], frac=1.0)
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    for b, name in ((0, "cfg2"), (1, "cfg2_scan1")):
        d = np.load(os.path.join(golden, "%s_reference.npz" % name))
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(y[b], np.float32).tobytes())
        h.update(np.ascontiguousarray(lam[b], np.float32).tobytes())
        assert str(d["digest"]) == h.hexdigest(), name
        assert abs(float(d["sigma_x"]) - sx) <= 1e-9 * sx, name
        assert float(d["kkt"]) < 1e-9, name
