"""Host logic of bench.py that needs no GPU: the self-launch of N ranks
(`bench.py --gpus N` started without torchrun), the rendezvous port, and the
rank environment every rank reads."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_launcher_command():
    cmd = bench.launcher_cmd(["--gpus", "4", "--steps", "7"], 4, 29511)
    assert cmd[:3] == [sys.executable, "-m", "torch.distributed.run"]
    assert "--nnodes=1" in cmd and "--nproc-per-node=4" in cmd
    assert "--master-addr=127.0.0.1" in cmd and "--master-port=29511" in cmd
    i = cmd.index(os.path.abspath(bench.__file__))
    assert cmd[i + 1:] == ["--gpus", "4", "--steps", "7"]


def test_free_port_is_bindable():
    p = bench.free_port()
    assert 0 < p < 65536
    s = socket.socket()
    try:
        s.bind(("127.0.0.1", p))
    finally:
        s.close()


def test_rank_environment(monkeypatch):
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("LOCAL_RANK", "3")
    assert bench.dist_env() == (3, 4, 3)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k)
    assert bench.dist_env() == (0, 1, 0)


@pytest.mark.timeout(180)
def test_launcher_starts_ranks_with_their_environment(tmp_path):
    """The launch command, with the benchmark swapped for a stand-in script,
    starts 2 local ranks that each see their own RANK and WORLD_SIZE."""
    out = tmp_path / "ranks"
    out.mkdir()
    script = tmp_path / "rank.py"
    script.write_text(
        "import os, pathlib\n"
        f"d = pathlib.Path({str(out)!r})\n"
        "(d / os.environ['RANK']).write_text(os.environ['WORLD_SIZE'] + ' ' + "
        "os.environ['LOCAL_RANK'])\n")
    cmd = bench.launcher_cmd([], 2, bench.free_port())
    cmd = cmd[:-1] if cmd[-1] == os.path.abspath(bench.__file__) else cmd
    cmd.append(str(script))
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=170)
    assert r.returncode == 0, r.stderr[-2000:]
    got = {p.name: p.read_text() for p in out.iterdir()}
    assert got == {"0": "2 0", "1": "2 1"}, json.dumps(got)
