"""Host-side check of the two-lane tile's shared-memory layout (the
constants are read from kernels_pair.cuh): the two transposes move every
value to the right lane, stay inside the per-warp buffer, and every
16-byte access pattern hits 8 distinct bank groups in each quarter warp
(the unit a 16-byte shared access is served in)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = open(os.path.join(ROOT, "paper_1306_1373_gb300", "csrc", "kernels_pair.cuh")).read()


def const(name):
    return int(re.search(r"constexpr int %s = (\d+);" % name, HDR).group(1))


S, L = const("kXSlot"), const("kXRowHalf")
BLOCKS = 16
XBYTES = BLOCKS * S


def write_addr(k, h, j, q):      # lane (k, h) stores row 4h + j, column quad q
    return k * S + h * L + j * 32 + q * 16


def read_addr(k, h, r):          # lane (k, h) loads row r, its column quad h
    return k * S + (r >> 2) * L + (r & 3) * 32 + h * 16


def lanes():
    return [(lane >> 1, lane & 1) for lane in range(32)]


def conflict_free(addrs):
    for quarter in range(4):
        groups = [(a // 16) % 8 for a in addrs[8 * quarter:8 * quarter + 8]]
        if len(set(groups)) != 8:
            return False
    return True


def test_transpose_accesses_are_conflict_free_and_in_bounds():
    for j in range(4):
        for q in range(2):
            addrs = [write_addr(k, h, j, q) for k, h in lanes()]
            assert conflict_free(addrs) and max(addrs) + 16 <= XBYTES
    for r in range(8):
        addrs = [read_addr(k, h, r) for k, h in lanes()]
        assert conflict_free(addrs) and max(addrs) + 16 <= XBYTES


def test_transpose_moves_rows_into_column_quads():
    mem = {}
    for k, h in lanes():                       # row pass output: lane h holds rows 4h..4h+3
        for j in range(4):
            for q in range(2):
                for t in range(4):
                    mem[write_addr(k, h, j, q) + 4 * t] = (k, 4 * h + j, 4 * q + t)
    assert len(mem) == BLOCKS * 64             # no two values share a word
    for k, h in lanes():                       # column pass input: lane h holds columns 4h..4h+3
        for r in range(8):
            for t in range(4):
                assert mem[read_addr(k, h, r) + 4 * t] == (k, r, 4 * h + t)


def test_sample_slots_are_conflict_free():
    park = XBYTES
    for half in range(2):
        addrs = [park + lane * 32 + 16 * (half ^ ((lane >> 2) & 1)) for lane in range(32)]
        assert conflict_free(addrs)
