"""Block admission of the serving loop (csrc/admission.h), host logic only.

Every served request is one cooperative grid whose blocks must all be
resident together.  The server fixes each request's launch shape when it is
submitted and admits it only if its blocks are sure to fit next to the
running grids.  These tests compile the admission header with g++ and check,
on a simulated 152-SM device, that every admitted set of grids can be placed
even when the hardware spreads the small blocks as badly as it can, and that
two mid-size requests whose one-block-per-SM grids together exceed the SM
count are never admitted together."""
import ctypes
import random
import subprocess

import pytest

from tests.test_host_logic import CSRC

SMS, PER = 152, 3


@pytest.fixture(scope="module")
def adm(tmp_path_factory):
    d = tmp_path_factory.mktemp("adm")
    src = d / "adm.cpp"
    src.write_text(
        '#include "admission.h"\n'
        'using namespace nnqp;\n'
        'extern "C" void shape(long long slices, int sms, int per, int share, int* cls, int* tpb, int* blocks) {'
        ' RequestShape r = request_shape(slices, sms, per, share); *cls = r.cls; *tpb = r.tpb; *blocks = r.blocks; }\n'
        'extern "C" int can_admit(int sms, int per, int full, int small, int cls, int blocks) {'
        ' BlockLedger L; L.sms = sms; L.small_per_sm = per; L.full_in_use = full; L.small_in_use = small;'
        ' RequestShape r; r.cls = cls; r.blocks = blocks; return L.can_admit(r) ? 1 : 0; }\n')
    so = d / "adm.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)])
    L = ctypes.CDLL(str(so))
    ip = ctypes.POINTER(ctypes.c_int)
    L.shape.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip, ip]
    L.can_admit.argtypes = [ctypes.c_int] * 6
    return L


def shape(adm, nodes, share=0):
    c, t, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    adm.shape((nodes + 31) // 32, SMS, PER, share, ctypes.byref(c), ctypes.byref(t), ctypes.byref(b))
    return c.value, t.value, b.value


def test_request_shapes_follow_the_single_system_sizing(adm):
    assert shape(adm, 5_000) == (0, 256, 20)          # 157 slices: small 256-thread grid
    assert shape(adm, 32_000) == (1, 512, 125)        # 1000 slices: one 512-thread block per SM, 125 SMs
    assert shape(adm, 150_000) == (1, 512, 152)       # up to 32 slices per SM: every SM
    assert shape(adm, 1_000_000) == (0, 256, SMS * PER)   # whole co-resident grid: runs alone
    assert shape(adm, 32_000, share=40) == (1, 512, 40)


def test_two_mid_size_requests_are_not_admitted_together(adm):
    """Two 32k-node requests take 125 whole SMs each: 250 > 152, so the second
    waits (counting both as 125 of 456 small-block units would admit both, and
    the second grid could not become resident)."""
    cls, _, b = shape(adm, 32_000)
    assert cls == 1 and b == 125
    assert adm.can_admit(SMS, PER, 0, 0, cls, b)
    assert not adm.can_admit(SMS, PER, b, 0, cls, b)
    assert 2 * b <= SMS * PER   # the old sum-of-blocks rule would have admitted it


def test_whole_device_request_runs_alone(adm):
    cls, _, b = shape(adm, 1_000_000)
    assert adm.can_admit(SMS, PER, 0, 0, cls, b)
    assert not adm.can_admit(SMS, PER, 0, 1, cls, b)
    assert not adm.can_admit(SMS, PER, 1, 0, cls, b)
    assert not adm.can_admit(SMS, PER, 0, b, 0, 1)


def place(sm_state, cls, blocks):
    """Adversarial placement: SMALL blocks go one per SM onto the emptiest
    SMs first (as many SMs touched as possible, which leaves the fewest empty
    SMs for whole-SM blocks); a FULL block needs an SM with nothing on it.
    Returns False if some block finds no room."""
    for _ in range(blocks):
        if cls == 1:
            k = next((i for i, s in enumerate(sm_state) if s == 0), None)
            if k is None:
                return False
            sm_state[k] = -1
        else:
            free = [i for i, s in enumerate(sm_state) if 0 <= s < PER]
            if not free:
                return False
            k = min(free, key=lambda i: sm_state[i])
            sm_state[k] += 1
    return True


def test_every_admitted_set_of_grids_is_co_resident_under_adversarial_placement(adm):
    rng = random.Random(2015)
    for trial in range(200):
        sm_state = [0] * SMS      # -1: a whole-SM block; k >= 0: k small blocks
        full = small = 0
        running = []
        for _ in range(40):
            if running and rng.random() < 0.4:
                # release a random running grid (its blocks leave their SMs)
                cls, b, where = running.pop(rng.randrange(len(running)))
                for k in where:
                    if cls == 1:
                        sm_state[k] = 0
                    else:
                        sm_state[k] -= 1
                if cls == 1:
                    full -= b
                else:
                    small -= b
                continue
            nodes = int(10 ** rng.uniform(3, 5.6))
            cls, _, b = shape(adm, nodes)
            if not adm.can_admit(SMS, PER, full, small, cls, b):
                continue
            before = list(sm_state)
            assert place(sm_state, cls, b), (trial, cls, b, full, small)
            where = [k for k in range(SMS) for _ in range(abs(sm_state[k] - before[k]))]
            running.append((cls, b, where))
            if cls == 1:
                full += b
            else:
                small += b
            assert small <= PER * (SMS - full)
