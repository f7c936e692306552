"""Client processes and the scheduler server on the CPU: the library's
client calls against the library's server logic over a byte-counting FIFO
engine (a test harness; the product serves the device engine). Failures are
made on the host: a client process that is killed, one that closes its
connection and keeps running, a malformed message. No GPU is involved."""
import ctypes
import os
import socket
import tempfile

import pytest

from paper_1712_04495_b300 import abi
from server_clients import Client, build_harness, wait_until

NO_TIMEOUT = abi.NO_TIMEOUT
MS = 1_000_000


@pytest.fixture(scope="module")
def harness_lib():
    d = tempfile.mkdtemp(prefix="sg_harness_")
    so = build_harness(d)
    L = ctypes.CDLL(so)
    L.harness_start.restype = ctypes.c_void_p
    L.harness_start.argtypes = [ctypes.c_char_p, ctypes.c_uint64]
    L.harness_counters.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.harness_used.restype = ctypes.c_uint64
    L.harness_used.argtypes = [ctypes.c_void_p]
    L.harness_stop.argtypes = [ctypes.c_void_p]
    return L


class Fake:
    def __init__(self, L, pool):
        self.L = L
        self.dir = tempfile.mkdtemp(prefix="sg_srv_")
        self.path = os.path.join(self.dir, "sock")
        self.h = L.harness_start(self.path.encode(), pool)
        assert self.h

    def counters(self):
        c = abi.SgServerCounts()
        self.L.harness_counters(self.h, ctypes.byref(c))
        return c.as_dict()

    def used(self):
        return self.L.harness_used(self.h)

    def stop(self):
        self.L.harness_stop(self.h)


@pytest.fixture
def server(harness_lib):
    s = Fake(harness_lib, 1000)
    yield s
    s.stop()


def test_declare_wait_release(server):
    a = Client(server.path)
    assert a.call("connect") == (1000, 1)
    t = a.call("declare", 600, 0, NO_TIMEOUT)
    assert a.call("wait", t, 2000 * MS) == (abi.SG_OK, 0)
    assert server.used() == 600
    assert a.call("release", t, 200) == abi.SG_OK              # partial post-free
    assert wait_until(lambda: server.used() == 400)
    assert a.call("release", t, 0) == abi.SG_OK
    assert wait_until(lambda: server.used() == 0)
    assert a.call("release", t, 0) == abi.SG_ERR_INVALID       # not held any more
    a.call("close")
    a.exit()
    c = server.counters()
    assert c["declares"] == 1 and c["grants"] == 1 and c["releases"] == 2
    assert wait_until(lambda: server.counters()["clients_reaped"] == 1)


def test_grant_is_pushed_to_a_waiting_client(server):
    a, b = Client(server.path), Client(server.path)
    a.call("connect")
    b.call("connect")
    ta = a.call("declare", 600, 0, NO_TIMEOUT)
    assert a.call("wait", ta, 2000 * MS)[0] == abi.SG_OK
    tb = b.call("declare", 600, 0, NO_TIMEOUT)
    assert b.call("wait", tb, 50 * MS) == (abi.SG_NOT_READY, None)
    assert a.call("release", ta, 0) == abi.SG_OK                # wake-on-release
    assert b.call("wait", tb, 5000 * MS)[0] == abi.SG_OK
    b.call("release", tb, 0)
    a.exit()
    b.exit()


def test_killed_client_is_reaped_and_its_memory_notifies_a_waiter(server):
    a, b = Client(server.path), Client(server.path)
    a.call("connect")
    b.call("connect")
    ta = a.call("declare", 700, 0, NO_TIMEOUT)
    assert a.call("wait", ta, 2000 * MS)[0] == abi.SG_OK
    tb = b.call("declare", 700, 0, NO_TIMEOUT)
    assert b.call("try", tb) == (abi.SG_NOT_READY, None)
    a.kill()                                                   # dies holding its grant
    assert b.call("wait", tb, 10_000 * MS)[0] == abi.SG_OK
    c = server.counters()
    assert c["clients_reaped"] == 1
    b.call("release", tb, 0)
    b.exit()


def test_killed_client_with_a_waiting_request_is_withdrawn(server):
    a, b = Client(server.path), Client(server.path)
    a.call("connect")
    b.call("connect")
    tb = b.call("declare", 700, 0, NO_TIMEOUT)
    assert b.call("wait", tb, 2000 * MS)[0] == abi.SG_OK
    a.call("declare", 700, 0, NO_TIMEOUT)                       # queued behind b
    a.kill()
    assert wait_until(lambda: server.counters()["clients_reaped"] == 1)
    assert b.call("release", tb, 0) == abi.SG_OK
    assert wait_until(lambda: server.used() == 0)              # nothing granted to the dead client
    c = server.counters()
    assert c["grants"] == 1 and c["tickets_open"] == 0
    b.exit()


def test_closed_connection_keeps_grants_until_the_process_exits(server):
    a, b = Client(server.path), Client(server.path)
    a.call("connect")
    b.call("connect")
    ta = a.call("declare", 700, 0, NO_TIMEOUT)
    assert a.call("wait", ta, 2000 * MS)[0] == abi.SG_OK
    a.call("close")                                            # abandoned, process still alive
    tb = b.call("declare", 700, 0, NO_TIMEOUT)
    assert b.call("wait", tb, 300 * MS) == (abi.SG_NOT_READY, None)
    assert server.counters()["clients_reaped"] == 0
    a.exit()                                                   # now the process is gone
    assert b.call("wait", tb, 10_000 * MS)[0] == abi.SG_OK
    b.exit()


def test_timeout_withdraws_a_waiting_request(server):
    a, b = Client(server.path), Client(server.path)
    a.call("connect")
    b.call("connect")
    ta = a.call("declare", 700, 0, NO_TIMEOUT)
    assert a.call("wait", ta, 2000 * MS)[0] == abi.SG_OK
    tb = b.call("declare", 700, 0, 50 * MS)
    assert b.call("wait", tb, 5000 * MS) == (abi.SG_ERR_TIMEOUT, None)
    assert server.counters()["timeouts"] == 1
    a.call("release", ta, 0)
    tb2 = b.call("declare", 700, 0, 50 * MS)                    # fits now
    assert b.call("wait", tb2, 5000 * MS)[0] == abi.SG_OK
    a.exit()
    b.exit()


def test_oversize_and_foreign_tickets(server):
    a, b = Client(server.path), Client(server.path)
    a.call("connect")
    b.call("connect")
    with pytest.raises(RuntimeError, match="code 3"):           # SG_ERR_TOO_LARGE
        a.call("declare", 5000, 0, NO_TIMEOUT)
    ta = a.call("declare", 100, 0, NO_TIMEOUT)
    assert a.call("wait", ta, 2000 * MS)[0] == abi.SG_OK
    assert b.call("release", ta, 0) == abi.SG_ERR_INVALID      # not b's grant
    assert a.call("release", ta, 0) == abi.SG_OK
    a.exit()
    b.exit()


def test_malformed_message_drops_only_that_connection(server):
    s = socket.socket(socket.AF_UNIX, socket.SOCK_SEQPACKET)
    s.connect(server.path)
    s.send(b"\x01\x02\x03")                                    # wrong size
    assert wait_until(lambda: server.counters()["protocol_errors"] == 1)
    s.close()
    a = Client(server.path)
    a.call("connect")
    t = a.call("declare", 10, 0, NO_TIMEOUT)
    assert a.call("wait", t, 2000 * MS)[0] == abi.SG_OK
    a.exit()
