"""bench.py's run records (no GPU): the JSON line printed once, and appended with a
hash of its workload and configuration to a JSONL file when asked."""
import json


def test_jsonl_record_and_config_hash(tmp_path, capsys):
    import bench
    path = str(tmp_path / "runs.jsonl")
    a = {"metric": "m", "value": 1.0, "config": {"workload": "w", "n_ch": 120}, "n_gpus": 1, "dtype": "f32"}
    b = dict(a, value=2.0)                               # another run of the same configuration
    c = dict(a, config={"workload": "w", "n_ch": 40})    # another configuration
    for line in (a, b, c):
        bench.emit(line, path)
    printed = [json.loads(x) for x in capsys.readouterr().out.splitlines()]
    assert printed == [a, b, c]
    recs = [json.loads(x) for x in open(path)]
    assert [r["value"] for r in recs] == [1.0, 2.0, 1.0]
    assert recs[0]["config_hash"] == recs[1]["config_hash"] != recs[2]["config_hash"]
    bench.emit(a, None)                                  # without a path nothing is written
    assert len(open(path).readlines()) == 3


def test_host_cpu_is_named():
    import bench
    name = bench.host_cpu()
    assert isinstance(name, str) and name and name != "unknown"
