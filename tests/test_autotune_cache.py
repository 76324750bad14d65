"""The FFT geometry cache file parser (host only): valid lines load, malformed ones are skipped."""
from paper_2010_06697_gb300 import build, rve


def test_cache_file_parser(tmp_path):
    build.build()
    import json
    p = tmp_path / "geo.jsonl"

    def line(dim, n, prec, half, full, **kw):
        d = {"kind": "rve-fft-geometry", "dim": dim, "n": n, "precision": prec, "lpb": 16, "tk64": 8,
             "tk32": 16, "rad_half": half, "rad_full": full, "ms": 0.1}
        d.update(kw)
        return json.dumps(d) + "\n"

    p.write_text(line(3, 128, 1, [8, 8], [8, 8, 2])
                 + line(3, 128, 1, [8, 4], [8, 8, 2])        # radices do not multiply to N/2
                 + "garbage\n"
                 + line(3, 128, 1, [8, 8], [8, 8, 2], tk64=999)  # tile wider than N/2
                 + line(2, 48, 0, [8, 3], [8, 2, 3], ms=0.2))
    assert rve.rve_autotune_load(str(p)) == 2
    # every line the file holds is JSON
    for ln in p.read_text().splitlines():
        if ln != "garbage":
            json.loads(ln)
    assert rve.rve_autotune_load(str(tmp_path / "missing.txt")) == rve.RVE_E_NOT_FOUND
