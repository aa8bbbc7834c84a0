"""Host-side check of the shared-memory layout that k_m2l_stage uses (restated here from its
definition; no GPU): the 243 bulk-copy runs of each parity class cover the class's 9x9x9
lattice exactly once, each run is a contiguous row range of one neighbour subgrid in the
parity-major cell order, every target's read at every stencil entry lands on the lattice cell
of its partner, and the 8 lanes of each quarter warp read 16-byte words on 8 distinct bank
groups for both record widths (20 and 28 floats).  The stencils come from the library."""
import numpy as np
import pytest

from paper_2101_08226_gb300 import api

SX, SY = 84, 9                     # lattice strides in cells
N_CELLS = 8 * SX + 8 * SY + 9      # cells in one class buffer


def cidx(a, b, c):
    return ((((a & 1) << 2) | ((b & 1) << 1) | (c & 1)) << 6) | ((a >> 1) << 4) | ((b >> 1) << 2) | (c >> 1)


def class_runs(cl):
    rx, ry, rz = (cl >> 2) & 1, (cl >> 1) & 1, cl & 1
    owner = {}
    for j in range(243):
        lx, ly, run = j // 27, (j // 3) % 9, j % 3
        x, y = 2 * lx + rx - 5, 2 * ly + ry - 5
        z1, z2 = (2, 6) if rz else (3, 7)
        lz0, lz1 = [(0, z1), (z1, z2), (z2, 9)][run]
        z = 2 * lz0 + rz - 5
        slot = ((x >> 3) + 1) * 9 + ((y >> 3) + 1) * 3 + ((z >> 3) + 1)
        row = cidx(x & 7, y & 7, z & 7)
        for k in range(lz1 - lz0):
            cell = lx * SX + ly * SY + lz0 + k
            zz = 2 * (lz0 + k) + rz - 5
            assert 0 <= cell < N_CELLS and cell not in owner
            assert ((zz >> 3) + 1) == ((z >> 3) + 1)           # the run stays in one neighbour
            assert row + k == cidx(x & 7, y & 7, zz & 7)        # consecutive rows
            owner[cell] = (slot, (x, y, zz))
    return owner


def test_runs_cover_each_class_once():
    for cl in range(8):
        assert len(class_runs(cl)) == 729


@pytest.mark.parametrize("theta", [0.34, 0.5, 0.7])
def test_every_read_lands_on_its_partner(theta):
    owners = [class_runs(cl) for cl in range(8)]
    for p in range(8):
        px, py, pz = (p >> 2) & 1, (p >> 1) & 1, p & 1
        for dx, dy, dz in api.stencil(theta, p).reshape(-1, 3):
            hx, hy, hz = px + dx + 5, py + dy + 5, pz + dz + 5
            assert min(hx, hy, hz) >= 0 and max(hx, hy, hz) <= 11
            cl = ((hx & 1) << 2) | ((hy & 1) << 1) | (hz & 1)
            off = (hx >> 1) * SX + (hy >> 1) * SY + (hz >> 1)
            for ia in range(4):
                for ib in range(4):
                    for ic in range(4):
                        _, xyz = owners[cl][ia * SX + ib * SY + ic + off]
                        assert xyz == (2 * ia + px + dx, 2 * ib + py + dy, 2 * ic + pz + dz)


@pytest.mark.parametrize("width", [20, 28])
def test_quarter_warps_hit_distinct_bank_groups(width):
    for half in range(2):
        for q in range(4):
            groups = {((width // 4) * (((half << 1) | ((lane >> 2) & 1)) * SX + (lane >> 3) * SY + (lane & 3))) % 8
                      for lane in range(8 * q, 8 * q + 8)}
            assert len(groups) == 8
