"""CPU checks of the host logic that cuts a (signal, scale) row into work items (csrc/work_plan.h,
shared by the plan and the allocation-free entry point). The header is compiled into a small host
harness with nvcc (no GPU needed) and its decomposition is checked, over seeded random rows, against
what the scan kernels rely on:

- the segments' stored ranges [t_out, t_end) tile the row's stored outputs exactly once, in order;
- each segment restarts 2L positions before its first output (t_dom = max(0, t_out - 2L)) from a
  first processed position t_a <= t_dom whose input element is 32-byte aligned, less than one
  alignment unit below t_dom;
- a window segment's sub-tiles cover [t_a, t_end) with none to spare, and its prologue stays within
  the bound the policy states; a chained segment's tiles are consecutive with consecutive status
  slots that all name the segment's first slot;
- rows go to window segments exactly when 2L <= 2T and the policy is not the one-chain-per-row one;
- the counting pass (no output array) agrees with the filling pass.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2110_11866_gb300", "csrc")

SEG_RESTART, SEG_ROW, SEG_PLAIN = 0, 1, 2
T = 256 * 16     # CTA tile: threads x items
WT = 32 * 16     # warp-tile

HARNESS = r"""
#include "work_plan.h"
using namespace msft;
// fields per item: t_a, t_dom, t_out, t_end, n_sub, slot, slot_first, x_off, n, out_off, chain
extern "C" long long row_work_c(long long N, long long L, long long D, long long x_off, long long out_off,
                                int align, int policy, int chain, long long wt, int warp_window,
                                long long o_lo, long long o_hi, long long T, long long* fields, long long cap,
                                long long* slots, long long* subtiles, int* chained) {
  RowSpec r{N, L, D, x_off, out_off, 0, align, policy, chain, wt, warp_window, o_lo, o_hi};
  bool ch = false;
  long long sl = *slots, st = 0;
  const long long n = row_work(r, T, nullptr, &sl, &st, &ch);
  if (fields == nullptr || n > cap) {
    *slots = sl;
    *subtiles = st;
    *chained = ch ? 1 : 0;
    return n;
  }
  WorkItem* w = new WorkItem[n > 0 ? n : 1];
  st = 0;
  const long long m = row_work(r, T, w, slots, &st, &ch);
  for (long long i = 0; i < m; ++i) {
    long long* f = fields + 11 * i;
    f[0] = w[i].t_a; f[1] = w[i].t_dom; f[2] = w[i].t_out; f[3] = w[i].t_end; f[4] = w[i].n_sub;
    f[5] = w[i].slot; f[6] = w[i].slot_first; f[7] = w[i].x_off; f[8] = w[i].n; f[9] = w[i].out_off;
    f[10] = w[i].chain;
  }
  delete[] w;
  *subtiles = st;
  *chained = ch ? 1 : 0;
  return m;
}
extern "C" void ss_window_tiles_c(long long t_grid, long long kb, long long L, int horner, long long tile,
                                  long long* a, long long* b) {
  ss_window_tiles(t_grid, kb, L, horner != 0, tile, a, b);
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("work_plan")
    src = d / "harness.cu"
    src.write_text(HARNESS)
    so = d / "libwork_plan_harness.so"
    cmd = [nvcc, "-std=c++17", "-O1", "-shared", "-Xcompiler", "-fPIC", "-gencode",
           "arch=compute_103a,code=sm_103a", "-I", CSRC, str(src), "-o", str(so)]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(str(so))
    f = lib.row_work_c
    ll, i32, pll, pi = ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int)
    f.restype = ll
    f.argtypes = [ll, ll, ll, ll, ll, i32, i32, i32, ll, i32, ll, ll, ll, pll, ll, pll, pll, pi]
    g = lib.ss_window_tiles_c
    g.restype = None
    g.argtypes = [ll, ll, ll, i32, ll, pll, pll]
    f.window_tiles = g
    return f


def run(f, N, L, D, x_off, out_off, align, policy, wt, warp_window, o_lo=0, o_hi=0, slot0=0):
    slots = ctypes.c_longlong(slot0)
    sub = ctypes.c_longlong(0)
    ch = ctypes.c_int(0)
    n = f(N, L, D, x_off, out_off, align, policy, 7, wt, warp_window, o_lo, o_hi, T, None, 0,
          ctypes.byref(slots), ctypes.byref(sub), ctypes.byref(ch))
    n_count, sub_count, slots_count = n, sub.value, slots.value
    fields = np.zeros((max(n, 1), 11), dtype=np.int64)
    slots = ctypes.c_longlong(slot0)
    m = f(N, L, D, x_off, out_off, align, policy, 7, wt, warp_window, o_lo, o_hi, T,
          fields.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), n, ctypes.byref(slots),
          ctypes.byref(sub), ctypes.byref(ch))
    assert m == n_count and sub.value == sub_count and slots.value == slots_count
    return fields[:m], sub.value, slots.value, bool(ch.value)


def check_row(f, N, L, D, x_off, align, policy, warp_window, o_lo=0, o_hi=0, slot0=5):
    wt = WT if warp_window else T
    items, subtiles, slots_end, chained = run(f, N, L, D, x_off, 1000, align, policy, wt, warp_window,
                                              o_lo, o_hi, slot0)
    first, last = (o_lo, o_hi) if o_hi > 0 else (D, D + N)
    assert chained == (not (2 * L <= 2 * T and policy != SEG_PLAIN))
    # every item names the row
    assert np.all(items[:, 7] == x_off) and np.all(items[:, 8] == N) and np.all(items[:, 9] == 1000)
    assert np.all(items[:, 10] == 7)
    # segments, in order, partition [first, last)
    segs = []
    for it in items:
        key = (int(it[2]), int(it[3]))
        if not segs or segs[-1][0] != key:
            segs.append([key, []])
        segs[-1][1].append(it)
    pos = first
    for (t_out, t_end), its in segs:
        assert t_out == pos and t_end > t_out
        pos = t_end
    assert pos == last
    # restart point, alignment
    for (t_out, t_end), its in segs:
        for it in its:
            assert it[1] == max(0, t_out - 2 * L)
        t_a0 = int(its[0][0])
        t_dom = int(its[0][1])
        assert t_a0 <= t_dom and t_dom - t_a0 < align
        assert (x_off + t_a0) % align == 0
    total_sub = 0
    if not chained:
        assert np.all(items[:, 5] == -1) and np.all(items[:, 6] == -1)
        # window segments: one item per segment, sub-tiles cover [t_a, t_end) exactly
        sub = max(2 if warp_window else 1, -(-(16 if warp_window else 10) * L // wt))
        R = max(1, sub * wt - 2 * L - (align - 1))
        for (t_out, t_end), its in segs:
            assert len(its) == 1
            t_a, n_sub = int(its[0][0]), int(its[0][4])
            assert t_a + n_sub * wt >= t_end and t_a + (n_sub - 1) * wt < t_end
            assert t_end - t_out <= R
            total_sub += n_sub
        assert slots_end == slot0
    else:
        slot = slot0
        R = max(4 * T, 4 * L) if policy == SEG_RESTART else N
        for (t_out, t_end), its in segs:
            assert t_end - t_out <= max(R, 1)
            first_slot = slot
            for k, it in enumerate(its):
                assert it[0] == its[0][0] + k * T and it[4] == 1
                assert it[5] == slot and it[6] == first_slot
                slot += 1
            t_a = int(its[0][0])
            assert t_a + len(its) * T >= t_end and t_a + (len(its) - 1) * T < t_end
            total_sub += len(its)
        assert slots_end == slot
    assert subtiles == total_sub


@pytest.mark.parametrize("policy", [SEG_RESTART, SEG_ROW, SEG_PLAIN])
@pytest.mark.parametrize("warp_window", [0, 1])
def test_row_work_random_rows(harness, policy, warp_window):
    rng = np.random.default_rng(100 + 10 * policy + warp_window)
    for _ in range(300):
        N = int(rng.choice([1, 2, 7, 511, 512, 513, 4095, 4096, 4097]) if rng.random() < 0.3
                else rng.integers(1, 400000))
        L = int(np.exp(rng.uniform(np.log(1), np.log(60000))))
        D = L + int(rng.integers(0, 5))
        x_off = int(rng.integers(0, 1 << 20))
        align = int(rng.choice([4, 8]))
        check_row(harness, N, L, D, x_off, align, policy, warp_window)


def test_row_work_output_window(harness):
    """Rows of a padded (edge-extended) batch store only their centre [o_lo, o_hi)."""
    rng = np.random.default_rng(7)
    for _ in range(300):
        n = int(rng.integers(1, 200000))
        L = int(np.exp(rng.uniform(0, np.log(20000))))
        pad = L + int(rng.integers(0, 40))
        N = n + 2 * pad
        D = L + int(rng.integers(0, 3))
        o_lo = D + pad
        for policy in (SEG_RESTART, SEG_ROW, SEG_PLAIN):
            check_row(harness, N, L, D, int(rng.integers(0, 1 << 20)), 8, policy, 1, o_lo, o_lo + n)


def test_row_work_edges(harness):
    """Window lengths at the window-segment boundary (2L = 2T) and one-sample rows."""
    for L in (T - 1, T, T + 1):
        for policy in (SEG_RESTART, SEG_ROW, SEG_PLAIN):
            for N in (1, 3, T, 10 * T + 3):
                check_row(harness, N, L, L, 3, 8, policy, 1)
                check_row(harness, N, L, L, 0, 4, policy, 0)


def test_start_state_window_tiles(harness):
    """The tiles whose sums a start-state item reads (ss_window_tiles, the rule the plan uses to
    choose which tile sums to compute) are exactly the tiles that lie wholly inside the item's
    window [u0, t_a) and at or after the row's tile 0; with the masked sum of the part of the window
    in front of them (from max(u0, t_grid) to their start, inside one tile) they cover the window's
    positions from t_grid on exactly once. Brute force over seeded random rows, both window forms."""
    rng = np.random.default_rng(31)
    tile = 512
    a, b = ctypes.c_longlong(0), ctypes.c_longlong(0)
    for _ in range(3000):
        t_grid = -512 + int(rng.integers(0, 8))
        kb = int(rng.integers(1, 400))
        L = int(rng.choice([int(rng.integers(1, 300)), int(rng.integers(256, 50000))]))
        horner = int(rng.integers(0, 2))
        harness.window_tiles(t_grid, kb, L, horner, tile, ctypes.byref(a), ctypes.byref(b))
        t_a = t_grid + tile * kb
        u0 = t_a - 2 * L - horner
        full = [k for k in range(kb) if t_grid + tile * k >= u0 and t_grid + tile * (k + 1) <= t_a]
        assert b.value == kb and list(range(a.value, b.value)) == full, (t_grid, kb, L, horner)
        # the masked part [max(u0, t_grid), first full tile) lies inside one tile (the whole window
        # when no tile is full)
        lo = max(u0, t_grid)
        head_end = t_grid + tile * full[0] if full else t_a
        assert 0 <= head_end - lo < tile or (not full and head_end - lo == tile), (t_grid, kb, L, horner)
