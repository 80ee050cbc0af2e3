"""Cases run against the library built with invariant checks (LOB_CHECKED=1
selects it): every case must match the oracle bit-exactly and leave the
status word at 0, i.e. no invariant failed after any message.  Run by
test_gpu_checked.py in a subprocess (the library is loaded once per process)."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path[:0] = [HERE, os.path.dirname(HERE)]

import numpy as np  # noqa: E402
import torch  # noqa: E402

import lobgen  # noqa: E402
from engine_harness import assert_same, run_both  # noqa: E402
from test_extremes import _extreme_streams  # noqa: E402


def main():
    assert os.environ.get("LOB_CHECKED") == "1"
    import paper_2308_13289_b300 as eng
    from paper_2308_13289_b300 import _abi
    assert _abi.LIB_PATH.endswith("liblob_checked.so")
    n_cases = 0
    for cap in (1, 7, 100, 128, 250, 500, 512):
        for rule in (0, 1):
            msgs, off = lobgen.generate(lobgen.make_params(900 + cap + rule, "pm1"),
                                        [2000, 1, 0, 1999, 700, 64])
            g, r = run_both(msgs, off, cap, 2000, rule)
            assert_same(g, r)  # includes status == 0
            n_cases += 1
    for cap in (7, 300):
        msgs, off = _extreme_streams(8, 1500, 600 + cap)
        g, r = run_both(msgs, off, cap, 1500, 0)
        assert_same(g, r)
        n_cases += 1
    for cap in (100, 250):
        n_env, steps, per = 32, 20, 50
        m, _ = lobgen.generate(lobgen.make_params(70 + cap), [steps * per] * n_env)
        draws = lobgen.agent_draws(5, n_env, steps)
        e = eng.Engine(n_env, cap, 2048)
        env = eng.Env(e, n_steps=steps, msgs_per_step=per)
        env.run(eng.messages_to_device(m), steps * per, 0, steps,
                torch.from_numpy(draws.view(np.int32)).cuda())
        _, st = e.stats()
        torch.cuda.synchronize()
        assert int(st.item()) == 0, int(st.item())
        n_cases += 1
    # the checks are live: a book loaded crossed (lob_set_book checks each
    # side's order, not the two sides against each other) is reported after
    # the next message, a padding record, without any fault
    e = eng.Engine(1, 8, 16)
    bk = {k: torch.full((1, 2, 8), -1, dtype=torch.int32, device="cuda")
          for k in ("price", "qty", "oid", "tid")}
    bk["time_ns"] = torch.full((1, 2, 8), -1, dtype=torch.int64, device="cuda")
    bk["count"] = torch.tensor([[1, 1]], dtype=torch.int32, device="cuda")
    for k, (b, a) in dict(price=(105, 100), qty=(5, 5), oid=(1, 2), tid=(0, 0)).items():
        bk[k][0, 0, 0], bk[k][0, 1, 0] = b, a
    bk["time_ns"][0, :, 0] = 0
    e.set_book(bk)
    pad = np.zeros(1, dtype=lobgen.MSG_DTYPE)
    e.process_batch(eng.messages_to_device(pad), torch.tensor([0, 1], dtype=torch.int64,
                                                              device="cuda"))
    _, st = e.stats()
    torch.cuda.synchronize()
    assert int(st.item()) & eng.STATUS_CHECK, int(st.item())
    e.close()
    print("checked-ok %d cases" % n_cases)


if __name__ == "__main__":
    main()
