"""The batched-launch autotuner on the GPU: it measures every group of a sample batch drawn
from the many-tables recipe, keeps a setting no slower than the defaults on that sample,
caches it per device and library build, and the tuned setting changes results within
rounding only: every table stays within 2e-6 of the oracle, tuned and default results agree
to 1e-6 (the FP32 partial sums are grouped differently), and a fixed setting reproduces its
bits."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2604_23826_gb300")
from paper_2604_23826_gb300 import inputs, tune  # noqa: E402


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mode", [G.STATS_BF16X3, G.STATS_BF16X4])
def test_autotune_sample_batch(tmp_path, mode):
    params = inputs.many_tables_shapes(3, 4096, n_hi=3e5)[:96]
    dev = torch.device("cuda")
    blocks, host = [], []
    for t, (n, p, mu, sd) in enumerate(params):
        ld = (n + 3) // 4 * 4
        blk = torch.empty((p, ld), dtype=torch.float32, device=dev)
        inputs.gen_table(torch, n, p, mu, sd, 7_000 + t, dev, out=blk[:, :n])
        blocks.append(blk)
        host.append(blk[:, :n].cpu().numpy())
    cols = [[b[j, :n] for j in range(p)] for b, (n, p, _, _) in zip(blocks, params)]
    rows = [n for n, _, _, _ in params]
    mk = lambda: [G.stats_init(G.Config([G.STATS_F32] * p, mode, [0] * p)) for _, p, _, _ in params]  # noqa: E731
    path = str(tmp_path / "tuning.json")

    def run(ctxs):
        G.stats_accumulate_batched(ctxs, cols, rows)
        return [G.stats_finalize(c).cov for c in ctxs]

    try:
        base = run(mk())
        entry = tune.autotune_batched(mk(), cols, rows, reps=2, workload="test", path=path, force=True)
        print(f"\nmode={mode}: {entry}")
        assert set(entry["choice"]) == {f"w{w}_{mode}" for w in (8, 16, 32, 64)}
        for m in entry["measured"].values():
            assert m["chosen_ms"] <= m["default_ms"]
        for name, t in entry["choice"].items():
            assert G.stats_get_batch_tuning(int(name.split("_")[0][1:]), mode) == t
        # cached: a second call returns the entry without measuring
        assert tune.autotune_batched(mk(), cols, rows, workload="test", path=path) == entry
        tuned = run(mk())
        again = run(mk())
        for t, X in enumerate(host):
            cov = O.cov_twopass_columns([X[j].astype(np.float64) for j in range(X.shape[0])])
            assert rel_fro(tuned[t], cov) < 2e-6 and rel_fro(base[t], cov) < 2e-6, t
            assert rel_fro(tuned[t], base[t]) < 1e-6, t
            assert np.array_equal(tuned[t], again[t]), t
    finally:
        for w in (8, 16, 32, 64):
            G.stats_set_batch_tuning(w, mode, tune.DEFAULT)
