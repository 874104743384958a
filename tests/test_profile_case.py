"""The profiling entry point parses its cases on a CPU-only machine (nothing is launched)."""
import pytest

from paper_1109_2935_gb300 import profile_case


def test_help_and_case_names(capsys):
    with pytest.raises(SystemExit) as e:
        profile_case.main(["--help"])
    assert e.value.code == 0
    text = capsys.readouterr().out
    for case in ("batch", "ptc", "wilson", "schwarz"):
        assert case in text


def test_unknown_case_is_rejected():
    with pytest.raises(SystemExit) as e:
        profile_case.main(["staggered"])
    assert e.value.code != 0


def test_algorithmic_bytes_per_site():
    # per site: 4 links (each link is read once over both parities), the input and output
    # spinors and the clover term; FP64-18: 4 x 144 + 192 + 192 + 576 = 1536
    assert profile_case.SITE_BYTES == {"f64": 1536, "f32": 672, "f16": 344}
