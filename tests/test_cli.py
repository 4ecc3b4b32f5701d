"""The command line's file handling and its calls into the library, on the
CPU: the graph class and the F1 function are replaced by fakes that record
what the command asks of them (the GPU path itself is covered by the parity
tests)."""
import io
import json

import numpy as np
import pytest

from paper_2210_03211_gb300 import cli


def test_edge_list_and_cover_files(tmp_path):
    p = tmp_path / "g.txt"
    p.write_text("# Undirected graph\n# FromNodeId\tToNodeId\n0\t1\n1 2\n% other comment\n7 0\n")
    src, dst = cli.read_edge_list(str(p))
    assert src.dtype == np.int32 and src.tolist() == [0, 1, 7] and dst.tolist() == [1, 2, 0]
    c = tmp_path / "c.txt"
    cli.write_cover(str(c), [np.array([3, 1, 2]), [5, 6]])
    assert c.read_text() == "3 1 2\n5 6\n"
    assert [x.tolist() for x in cli.read_cover(str(c))] == [[3, 1, 2], [5, 6]]
    bad = tmp_path / "bad.txt"
    bad.write_text("0 -4\n")
    with pytest.raises(ValueError):
        cli.read_edge_list(str(bad))


class FakeGraph:
    calls = []

    def __init__(self, src, dst):
        self.n, self.m = int(max(src.max(), dst.max()) + 1), int(src.shape[0])
        FakeGraph.calls.append(("create", src.tolist(), dst.tolist()))
        self.iteration = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        FakeGraph.calls.append(("close",))

    def autotune(self, q, trials):
        FakeGraph.calls.append(("autotune", q, trials))
        return {"trials": 24}

    def set_partition(self, cover):
        FakeGraph.calls.append(("set_partition", [c.tolist() for c in cover]))

    def community_list(self):
        return [np.array([0, 1, 2 + self.iteration]), np.array([5, 6])]

    def run(self, q, thr, iters, on_iteration=None):
        FakeGraph.calls.append(("run", q, thr, iters))
        for it in (1, 2):
            self.iteration = it
            if on_iteration is not None:
                on_iteration(it, 10.0 * it)

        class St:
            iterations, converged, wcc_initial = 2, True, 5.0
            wcc_history = np.array([10.0, 20.0])
        return St()


def test_command_writes_results_snapshots_and_summary(tmp_path):
    edges = tmp_path / "g.txt"
    edges.write_text("0 1\n1 2\n5 6\n")
    cover = tmp_path / "start.txt"
    cover.write_text("0 1 2\n")
    truth = tmp_path / "truth.txt"
    truth.write_text("0 1 2\n5 6\n")
    FakeGraph.calls = []
    seen = {}

    def fake_f1(detected, reference):
        seen["f1"] = ([c.tolist() for c in detected], [c.tolist() for c in reference])
        return 0.75, None

    args = cli.parse_args([str(edges), "--queue-size", "64", "--threshold", "0.05", "--max-iters", "7",
                           "--output", str(tmp_path / "out.txt"), "--every-iteration", str(tmp_path / "it"),
                           "--resume", str(cover), "--ground-truth", str(truth), "--autotune"])
    buf = io.StringIO()
    s = cli.run(args, graph_cls=FakeGraph, f1_fn=fake_f1, out=buf)
    assert [c[0] for c in FakeGraph.calls] == ["create", "autotune", "set_partition", "run", "close"]
    assert FakeGraph.calls[2] == ("set_partition", [[0, 1, 2]])
    assert FakeGraph.calls[3] == ("run", 64, 0.05, 7)
    assert (tmp_path / "it" / "iteration_1.txt").read_text() == "0 1 3\n5 6\n"
    assert (tmp_path / "it" / "iteration_2.txt").read_text() == "0 1 4\n5 6\n"
    assert (tmp_path / "out.txt").read_text() == "0 1 4\n5 6\n"
    assert seen["f1"] == ([[0, 1, 4], [5, 6]], [[0, 1, 2], [5, 6]])
    assert json.loads(buf.getvalue()) == s
    assert s["iterations"] == 2 and s["wcc"] == [10.0, 20.0] and s["communities"] == 2
    assert s["memberships"] == 5 and s["f1_vs_ground_truth"] == 0.75 and s["edges_in"] == 3


def test_command_without_a_gpu_fails_loudly(tmp_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2210_03211_gb300 import build, lazyfox
    build.build()
    edges = tmp_path / "g.txt"
    edges.write_text("0 1\n1 2\n")
    with pytest.raises(lazyfox.LazyFoxError):
        cli.run(cli.parse_args([str(edges)]), out=io.StringIO())
