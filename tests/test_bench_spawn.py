"""bench.py --gpus N outside torchrun launches its own N ranks (frame shards, no collective in
the data path, counters summed at the end).  On CPU the launcher is exercised with gloo ranks
that decode their shards with the oracle."""
import json
import sys
import textwrap
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402

RANK_SCRIPT = textwrap.dedent('''
    import json, sys
    sys.path.insert(0, {root!r})
    import torch.distributed as dist
    import bench
    from tests.test_shard import _counts, TOTAL
    from paper_1911_08868_gb300.shard import reduce_counters, shard_range

    rank, world, local = bench.dist_env()
    dist.init_process_group("gloo")
    lo, hi = shard_range(TOTAL, world, rank)
    job = reduce_counters(_counts(lo, hi))
    if rank == 0:
        print("RESULT " + json.dumps({{"n_gpus": world, **job}}), flush=True)
    dist.destroy_process_group()
''')


def test_needs_spawn_only_outside_torchrun(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.needs_spawn(2) and bench.needs_spawn(8)
    assert not bench.needs_spawn(1)
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert not bench.needs_spawn(2)


def test_main_relaunches_itself_for_several_gpus(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    seen = {}

    def fake_spawn(nproc, script, argv):
        seen.update(nproc=nproc, script=script, argv=list(argv))
        return 0

    monkeypatch.setattr(bench, "spawn_ranks", fake_spawn)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--gpus", "2", "--steps", "3", "--warmup", "3"])
    with pytest.raises(SystemExit) as e:
        bench.main()
    assert e.value.code == 0
    assert seen == {"nproc": 2, "script": str(ROOT / "bench.py"), "argv": ["--gpus", "2", "--steps", "3", "--warmup", "3"]}


def test_two_spawned_gloo_ranks_report_two_gpus_and_the_unsplit_counters(tmp_path, capfd, monkeypatch):
    from tests.test_shard import TOTAL, _counts

    monkeypatch.delenv("WORLD_SIZE", raising=False)
    script = tmp_path / "rank.py"
    script.write_text(RANK_SCRIPT.format(root=str(ROOT)))
    rc = bench.spawn_ranks(2, str(script), [])
    out = capfd.readouterr().out
    assert rc == 0, out
    lines = [ln for ln in out.splitlines() if ln.startswith("RESULT ")]
    assert len(lines) == 1                              # rank 0 alone prints
    got = json.loads(lines[0][len("RESULT "):])
    assert got.pop("n_gpus") == 2
    assert got == _counts(0, TOTAL)
