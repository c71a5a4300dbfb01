"""CPU tests of the request server's admission policy (csrc/admission.h, the
function the server's workers call under its lock), compiled here with g++
behind a C harness: arrival order, memory budget, slot count, and the bypass
limit that keeps a large request from waiting for ever behind small ones."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1605_07951_gb300", "csrc")

HARNESS = r"""
#include <cstdint>
#include "admission.h"
extern "C" int admit(int count, const uint64_t *bytes, const int *bypassed, uint64_t used,
                     uint64_t budget, int active, int slots, int max_bypass) {
    return rsrr::admit_index(
        count, [&](int q) { return (size_t)bytes[q]; }, [&](int q) { return bypassed[q]; },
        (size_t)used, (size_t)budget, active, slots, max_bypass);
}
"""
MAX_BYPASS = 8  # the server's limit (kMaxBypass)


@pytest.fixture(scope="module")
def admit(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("admission")
    h = d / "harness.cpp"
    h.write_text(HARNESS)
    so = d / "libadmit.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", SRC, str(h), "-o", str(so)],
                   check=True, capture_output=True, text=True)
    L = C.CDLL(str(so))
    L.admit.restype = C.c_int
    L.admit.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_int,
                        C.c_int]

    def call(bytes_, bypassed, used, budget, active, slots, max_bypass=MAX_BYPASS):
        b = np.asarray(bytes_, dtype=np.uint64)
        p = np.asarray(bypassed, dtype=np.int32)
        return L.admit(len(b), b.ctypes.data, p.ctypes.data, used, budget, active, slots, max_bypass)
    return call


def test_arrival_order_when_everything_fits(admit):
    assert admit([5, 1, 1], [0, 0, 0], used=0, budget=100, active=0, slots=4) == 0


def test_no_free_slot_admits_nothing(admit):
    assert admit([1], [0], used=0, budget=100, active=4, slots=4) == -1


def test_empty_queue(admit):
    assert admit([], [], used=0, budget=100, active=0, slots=4) == -1


def test_a_later_request_passes_one_that_does_not_fit(admit):
    assert admit([80, 30, 10], [0, 0, 0], used=75, budget=100, active=1, slots=4) == 2
    assert admit([80, 30, 10], [0, 0, 0], used=40, budget=100, active=1, slots=4) == 1


def test_exact_fit_and_overfull_budget(admit):
    assert admit([60], [0], used=40, budget=100, active=1, slots=4) == 0
    assert admit([61], [0], used=40, budget=100, active=1, slots=4) == -1
    assert admit([1], [0], used=120, budget=100, active=1, slots=4) == -1  # never wraps around


def test_bypass_limit_blocks_the_requests_behind(admit):
    assert admit([80, 10], [MAX_BYPASS - 1, 0], used=50, budget=100, active=1, slots=4) == 1
    assert admit([80, 10], [MAX_BYPASS, 0], used=50, budget=100, active=1, slots=4) == -1
    # a blocked head still goes as soon as it fits
    assert admit([80, 10], [MAX_BYPASS, 0], used=20, budget=100, active=1, slots=4) == 0


def simulate(admit, sizes, budget, slots, durations):
    """Event simulation of the worker loop: admit while possible, finish the
    request that ends first, repeat.  Returns admission order, peak bytes."""
    queue = list(range(len(sizes)))
    bypassed = [0] * len(sizes)
    running, used, t, order, peak = [], 0, 0.0, [], 0
    while queue or running:
        while True:
            q = admit([sizes[i] for i in queue], [bypassed[i] for i in queue], used, budget,
                      len(running), slots)
            if q < 0:
                break
            for e in queue[:q]:
                bypassed[e] += 1
            i = queue.pop(q)
            used += sizes[i]
            peak = max(peak, used)
            running.append((t + durations[i], i))
            order.append(i)
        assert running, "deadlock: nothing runs and nothing is admitted"
        running.sort()
        t, i = running.pop(0)
        used -= sizes[i]
    return order, peak, bypassed


def test_simulated_stream_respects_budget_and_never_starves(admit):
    rng = np.random.default_rng(11)
    budget, slots = 100, 4
    # one large request early in a long stream of small ones
    sizes = [int(s) for s in rng.integers(5, 30, 60)]
    sizes[3] = 95
    durations = [float(d) for d in rng.uniform(0.5, 2.0, 60)]
    order, peak, bypassed = simulate(admit, sizes, budget, slots, durations)
    assert sorted(order) == list(range(60))
    assert peak <= budget
    assert max(bypassed) <= MAX_BYPASS
    # the large request went after at most MAX_BYPASS later arrivals
    later_first = sum(1 for i in order[:order.index(3)] if i > 3)
    assert later_first <= MAX_BYPASS
    assert bypassed[3] == MAX_BYPASS == later_first  # the limit was what let it through
