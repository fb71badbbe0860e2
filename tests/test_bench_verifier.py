"""The bench's oracle process holds submitted jobs until it is started (the
host-driven timed sections run without the oracle beside them), then runs
the held ones and every later one as it is submitted; results come back in
any order of collection.  CPU only."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_jobs_are_held_until_start_then_run_as_submitted():
    v = bench.Verifier()
    try:
        a = v.submit(pow, 2, 10)
        b = v.submit(divmod, 17, 5)
        assert a.res is None and b.res is None and len(v.held) == 2  # nothing runs yet
        v.start()
        assert not v.held
        c = v.submit(max, 3, 9, 4)  # started: runs at once
        assert c.res is not None
        assert (c.get(), b.get(), a.get()) == (9, (3, 2), 1024)
    finally:
        v.close()


def test_get_starts_the_held_jobs():
    v = bench.Verifier()
    try:
        a = v.submit(pow, 3, 4)
        assert a.get() == 81 and v.running
    finally:
        v.close()
