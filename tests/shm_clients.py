"""Client processes for the shared-memory scheduler tests. A client runs the
commands the test sends over a pipe, so the test decides every step and can
kill a client between steps. Failures are made on the host: a killed
process, a process that dies holding the file lock, bytes of the segment
overwritten by the test."""
import fcntl
import mmap
import multiprocessing as mp
import os
import struct
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# fixed offsets of the segment (pinned by static_asserts in the library)
HDR_DIRTY, HDR_USED = 48, 64
TK_BASE, TK_SIZE = 384, 88
TK_PID, TK_NEED_G, TK_OFFSET = 8, 40, 48


def seg_path(name: str) -> str:
    return "/dev/shm" + name


def poke(name: str, offset: int, fmt: str, value) -> None:
    """Overwrite bytes of the segment (a test's stand-in for corruption)."""
    with open(seg_path(name), "r+b") as f:
        m = mmap.mmap(f.fileno(), 0)
        struct.pack_into(fmt, m, offset, value)
        m.close()


def peek(name: str, offset: int, fmt: str):
    with open(seg_path(name), "rb") as f:
        m = mmap.mmap(f.fileno(), 0, prot=mmap.PROT_READ)
        v = struct.unpack_from(fmt, m, offset)[0]
        m.close()
    return v


def _ofd_lock(fd: int) -> None:
    # struct flock {short l_type; short l_whence; off_t l_start; off_t l_len; pid_t l_pid;}
    F_OFD_SETLKW = 38
    fl = struct.pack("hhqqi4x", fcntl.F_WRLCK, os.SEEK_SET, 0, 1, 0)
    fcntl.fcntl(fd, F_OFD_SETLKW, fl)


def _worker(name, conn, gpu):
    sys.path.insert(0, ROOT)
    from paper_1712_04495_b300 import abi
    h = None
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
            if op == "open":
                h = abi.sg_shm_open(name, *cmd[1:])
                res = os.getpid()
            elif op == "declare":
                res = abi.sg_shm_declare(h, cmd[1], cmd[2])
            elif op == "wait":
                t0 = time.monotonic_ns()
                rc, g = abi.sg_shm_wait(h, cmd[1], cmd[2])
                res = (rc, g.offset if g else None, time.monotonic_ns() - t0)
            elif op == "try":
                rc, g = abi.sg_shm_try(h, cmd[1])
                res = (rc, g.offset if g else None)
            elif op == "release":
                res = abi.sg_shm_release(h, cmd[1], cmd[2])
            elif op == "close":
                abi.sg_shm_close(h)
                h = None
                res = 0
            elif op == "die_holding_lock":
                # take the segment's file lock, mark an update in progress,
                # damage the used-bytes count and end without unlocking
                fd = os.open(seg_path(name), os.O_RDWR)
                _ofd_lock(fd)
                poke(name, HDR_DIRTY, "<I", 1)
                poke(name, HDR_USED, "<Q", cmd[1])
                conn.send(("ok", 0))
                os._exit(0)
            elif op == "triad":
                # the triad job's layout on the grant: a, b, c at 0, 4n, 8n
                t, n, key = cmd[1], cmd[2], cmd[3]
                abi.sg_shm_pool(h)
                rc, g = abi.sg_shm_try(h, t)
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


class ShmClient:
    def __init__(self, name: str, gpu: bool = False):
        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe()
        self.proc = ctx.Process(target=_worker, args=(name, child, gpu), daemon=True)
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


def stress(name: str, seed: int, cycles: int, max_need: int, q) -> None:
    """declare -> wait -> hold -> release loops; reports every grant as
    (grant_ns, offset, need_g, released_before_ns)."""
    sys.path.insert(0, ROOT)
    import random
    from paper_1712_04495_b300 import abi
    rnd = random.Random(seed)
    h = abi.sg_shm_open(name)
    log = []
    try:
        for _ in range(cycles):
            need = rnd.randint(1, max_need)
            rc, t = abi.sg_shm_declare(h, need, rnd.randint(0, 2))
            assert rc == abi.SG_OK, rc
            rc, g = abi.sg_shm_wait(h, t, 30 * 10 ** 9)
            assert rc == abi.SG_OK, rc
            time.sleep(rnd.random() * 0.002)
            before = time.monotonic_ns()
            assert abi.sg_shm_release(h, t, 0) == abi.SG_OK
            log.append((g.grant_time_ns, g.offset, (need + 255) // 256 * 256, before))
        q.put(("done", log))
    except Exception as e:
        q.put(("error", repr(e)))
    finally:
        abi.sg_shm_close(h)
