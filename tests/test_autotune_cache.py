"""The FFT geometry cache file parser (host only): valid lines load, malformed ones are skipped."""
from paper_2010_06697_gb300 import build, rve


def test_cache_file_parser(tmp_path):
    build.build()
    p = tmp_path / "geo.txt"
    p.write_text("rve-fft-geometry 3 128 1 16 8 16 2 8 8 3 8 8 2 0.1\n"
                 "rve-fft-geometry 3 128 1 16 8 16 2 8 4 3 8 8 2 0.1\n"     # radices do not multiply to N/2
                 "garbage\n"
                 "rve-fft-geometry 2 48 0 32 8 16 2 8 3 3 8 2 3 0.2\n")
    assert rve.rve_autotune_load(str(p)) == 2
    assert rve.rve_autotune_load(str(tmp_path / "missing.txt")) == rve.RVE_E_NOT_FOUND
