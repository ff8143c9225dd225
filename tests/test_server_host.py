"""Host logic of the serving loop, without a GPU: the library's fake-executor mode
(NATBEM_SERVER_FAKE=1) runs no device work, so admission order, budget accounting, refusals,
timeouts and shutdown are checked on the CPU. Run in a child process so the environment
variable reaches the library before the server is created."""
import os
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import os, sys, time
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_2506_06190_gb300 import build
    build.build()
    import paper_2506_06190_gb300 as nb
    import synthetic as S

    def job(nt):
        V, F = S.ring_sphere(nt)
        return dict(V=V, F=F, k=1.0, neumann=np.ones(len(F), np.complex64))

    small = nb.nat_bem_required_bytes(2000, 1)
    # budget for exactly one 2000-triangle request at a time
    jobs = [job(2000) for _ in range(4)]
    big = job(100000)                             # needs more than the whole budget
    with nb.Server(small + 1, slots=4) as srv:
        tickets = [srv.submit(j) for j in jobs]
        huge = srv.submit(big)
        st = srv.wait(huge, 10000)[0]
        assert st == nb.NAT_BEM_ENOMEM, st
        # the first request runs ~20 ms: a zero timeout on the last one times out, then succeeds
        assert srv.wait(tickets[-1], 0)[0] == nb.NAT_BEM_ETIMEOUT
        res = [srv.wait(t, 10000) for t in tickets]
        assert all(r[0] == nb.NAT_BEM_OK for r in res)
        # one at a time under this budget: each waited for the previous ones (FIFO)
        queues = [r[5] for r in res]
        assert queues[0] < queues[1] < queues[2] < queues[3], queues
        assert srv.reserved() == 0
    # a budget for all four: they overlap
    with nb.Server(4 * small + 1, slots=4) as srv:
        tickets = [srv.submit(j) for j in jobs]
        res = [srv.wait(t, 10000) for t in tickets]
        assert all(r[0] == nb.NAT_BEM_OK for r in res)
        assert max(r[5] for r in res) < 15.0, [r[5] for r in res]   # none queued behind another
    print("ok")
""").replace("ROOT", repr(ROOT))


def test_server_admission_and_timeouts_on_host():
    env = dict(os.environ, NATBEM_SERVER_FAKE="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ok" in r.stdout


def test_server_create_needs_a_device_without_fake_mode():
    env = dict(os.environ)
    env.pop("NATBEM_SERVER_FAKE", None)
    code = textwrap.dedent("""
        import sys, ctypes
        sys.path.insert(0, ROOT)
        import paper_2506_06190_gb300 as nb
        h = ctypes.c_void_p()
        L = nb.lib()
        assert L.nat_bem_server_create(0, None, 2, ctypes.byref(h)) == nb.NAT_BEM_EINVAL
        assert L.nat_bem_server_create(1 << 30, None, 0, ctypes.byref(h)) == nb.NAT_BEM_EINVAL
        assert L.nat_bem_submit(None, None, None) == nb.NAT_BEM_EINVAL
        assert L.nat_bem_wait(None, 1, 0, None, None) == nb.NAT_BEM_EINVAL
        assert L.nat_bem_selftest_bounded_wait(0, None) == nb.NAT_BEM_EINVAL
        print("ok")
    """).replace("ROOT", repr(ROOT))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
