"""Client processes for the scheduler-server tests: each runs commands sent
by the test over a pipe, so the test decides every step, and a client can be
killed between steps (never with work of its own in flight)."""
import multiprocessing as mp
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_harness(out_dir: str) -> str:
    """The library's server over a byte-counting FIFO engine (no GPU)."""
    so = os.path.join(out_dir, "fake_server.so")
    src = os.path.join(ROOT, "tests", "server_harness", "fake_server.cpp")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-o", so, src, "-lpthread"])
    return so


def _worker(path, conn, gpu):
    sys.path.insert(0, ROOT)
    from paper_1712_04495_b300 import abi
    cl = None
    torch = None
    if gpu:
        import torch
        torch.cuda.set_device(0)
        torch.zeros(1, device="cuda")
    while True:
        cmd = conn.recv()
        op = cmd[0]
        try:
            if op == "exit":
                conn.send(("ok", os.getpid()))
                return
            if op == "connect":
                cl = abi.sg_client_connect(path)
                res = abi.sg_client_info(cl)
            elif op == "declare":
                need, prio, tmo = cmd[1], cmd[2], cmd[3]
                res = abi.sg_client_declare(cl, need, prio, tmo)
            elif op == "wait":
                rc, g = abi.sg_client_wait(cl, cmd[1], cmd[2])
                res = (rc, g.offset if g else None)
            elif op == "try":
                rc, g = abi.sg_client_try(cl, cmd[1])
                res = (rc, g.offset if g else None)
            elif op == "release":
                res = abi.sg_client_release(cl, cmd[1], cmd[2])
            elif op == "close":
                abi.sg_client_close(cl)
                cl = None
                res = 0
            elif op == "triad":
                # the triad job of Sec. "a5.1" layout on the grant: a, b, c at 0, 4n, 8n
                t, n, key = cmd[1], cmd[2], cmd[3]
                abi.sg_client_pool(cl)
                rc, g = abi.sg_client_try(cl, t)
                assert rc == abi.SG_OK and g.ptr
                a, b, c = g.ptr, g.ptr + 4 * n, g.ptr + 8 * n
                s = torch.cuda.Stream()
                out = torch.zeros(1, dtype=torch.int64, device="cuda")
                assert abi.sg_gen_triad(b, c, n, key, s.cuda_stream) == abi.SG_OK
                assert abi.sg_triad(a, b, c, 3.0, n, s.cuda_stream) == abi.SG_OK
                assert abi.sg_digest(a, n, out.data_ptr(), s.cuda_stream) == abi.SG_OK
                s.synchronize()                       # nothing of ours in flight after this
                res = (int(out.item()) & ((1 << 64) - 1), g.offset)
            else:
                raise ValueError(op)
            conn.send(("ok", res))
        except Exception as e:   # report to the test, keep serving
            conn.send(("err", repr(e)))


class Client:
    def __init__(self, path: str, gpu: bool = False):
        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe()
        self.proc = ctx.Process(target=_worker, args=(path, child, gpu), daemon=True)
        self.proc.start()

    def call(self, *cmd, timeout: float = 60.0):
        self.conn.send(cmd)
        if not self.conn.poll(timeout):
            raise TimeoutError(f"client did not answer {cmd}")
        status, res = self.conn.recv()
        if status != "ok":
            raise RuntimeError(res)
        return res

    def kill(self):
        self.proc.kill()
        self.proc.join(10)

    def exit(self):
        try:
            self.call("exit", timeout=10)
        finally:
            self.proc.join(10)


def wait_until(pred, timeout: float = 10.0, step: float = 0.01) -> bool:
    t0 = time.time()
    while time.time() - t0 < timeout:
        if pred():
            return True
        time.sleep(step)
    return pred()
