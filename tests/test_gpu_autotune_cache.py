"""The autotuner's persisted choices (WMG_AUTOTUNE_CACHE): a first process times the stencil's
launch shapes and appends its choice to the file; a second process reads it and launches the
same shape without timing (its report lists the cached entry)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json, sys
sys.path.insert(0, %r)
import torch
from paper_2505_14399_gb300 import _lib, api, synthetic
dims = (8, 8, 8, 8)
U = torch.from_numpy(synthetic.haar_links(dims, 1)).to(torch.complex64).cuda()
x = torch.from_numpy(synthetic.gaussian_rhs(dims, 2)).to(torch.complex64).cuda()
n0 = _lib.lib().mg_kernel_launches()
api.dslash(x, U, dims, 0.12)
torch.cuda.synchronize()
print(json.dumps({"launches": _lib.lib().mg_kernel_launches() - n0,
                  "report": json.loads(_lib.lib().mg_autotune_report().decode())}))
''' % ROOT


def _run(path):
    env = dict(os.environ, WMG_AUTOTUNE_CACHE=path)
    out = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True,
                         timeout=300, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_cache_file_round_trip(tmp_path):
    path = str(tmp_path / "tune.jsonl")
    first = _run(path)
    lines = [json.loads(l) for l in open(path)]
    assert len(lines) == 1 and lines[0]["volume"] == 8 ** 4 and lines[0]["nrhs"] == 1
    assert first["launches"] > 1                 # the shapes were timed, then the call launched
    times = lines[0]["all_ms"]                   # every candidate's time, the winner the fastest
    assert len(times) > 1 and times[lines[0]["variant"]] == min(times)
    second = _run(path)
    assert second["launches"] == 1               # read from the file: only the call itself
    assert second["report"][0]["variant"] == lines[0]["variant"] == first["report"][0]["variant"]
    assert len(open(path).readlines()) == 1      # nothing new appended
