"""The kernels' constants header is exactly what its generator writes: the
splits of pi/2, the words of 2/pi, the signed rows and the limits in
ptrig_constants.h come from gen_constants.py and nothing else edits them."""
import importlib.util
import os

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2502_10831_gb300", "csrc")


def test_header_matches_generator():
    spec = importlib.util.spec_from_file_location("gen_constants", os.path.join(CSRC, "gen_constants.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    with open(os.path.join(CSRC, "ptrig_constants.h")) as f:
        assert gen.main() == f.read()
