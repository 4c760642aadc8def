"""CPU model of the pooling kernel's bulk-copy staging (paper_2601_01210_gb300/csrc/k_pool_bp.cu):
for every work item of a set of image sizes, an item takes the staged path only when its copies
start on 16-byte boundaries with sizes that are multiples of 16 bytes and fit their buffers, and
every shared-memory word and byte the staged pooling reads lies inside the item's rows. The
buffer constants are read from the kernel's source, so a change there is checked here."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2601_01210_gb300", "csrc")


def constants():
    desc = open(os.path.join(CSRC, "desc.cuh")).read()
    src = open(os.path.join(CSRC, "k_pool_bp.cu")).read()
    threads = int(re.search(r"constexpr int kThreads = (\d+);", desc).group(1))
    assert re.search(r"constexpr int kPoolPerChunk = kThreads;", desc)
    per = threads
    seg = eval(re.search(r"constexpr int kPoolSegPx = ([^;]+);", src).group(1).replace("kPoolPerChunk", str(per)))
    zb = eval(re.search(r"constexpr int kPoolZBytes = ([^;]+);", src).group(1).replace("kPoolSegPx", str(seg)))
    cb = eval(re.search(r"constexpr int kPoolCBytes = ([^;]+);", src).group(1).replace("kPoolSegPx", str(seg)))
    return per, seg, zb, cb


def staged(W, H, J, I0, per, seg):
    """The kernel's eligibility test (pool_kernel's locate) for pooling factor 3, aligned frames."""
    Wc = (W + 2) // 3
    m = min(per, Wc - I0)
    n = min(seg, W - 3 * I0)
    return 3 * J + 3 <= H and n == 3 * m and n % 16 == 0, m, n


@pytest.mark.parametrize("W,H", [(1920, 1080), (1281, 721), (1280, 720), (960, 540), (640, 480), (48, 33),
                                 (768, 3), (769, 9), (16384, 64), (64, 16384), (3, 3), (1, 1)])
def test_staged_items_stay_in_bounds(W, H):
    per, seg, zbytes, cbytes = constants()
    assert zbytes % 16 == 0 and (zbytes + cbytes) % 16 == 0 and (3 * seg) % 16 == 0
    Wc, Hc = (W + 2) // 3, (H + 2) // 3
    segs = (Wc + per - 1) // per
    n_staged = 0
    for J in range(Hc):
        for sgi in range(segs):
            I0 = sgi * per
            ok, m, n = staged(W, H, J, I0, per, seg)
            if not ok:
                continue
            n_staged += 1
            x0 = 3 * I0
            # copies: three rows of 4n z-buffer bytes and 3n colour bytes, source offsets on 16 bytes
            # (the frame's base and pitches are checked by the kernel: bulk_ok)
            assert (4 * n) % 16 == 0 and (3 * n) % 16 == 0 and (4 * x0) % 16 == 0 and (3 * x0) % 16 == 0
            assert 4 * n <= 4 * seg and 3 * n <= 3 * seg            # each row inside its buffer row
            assert x0 + n <= W and 3 * J + 2 < H                    # the global rows and columns copied exist
            assert 3 * (4 * seg) <= zbytes and 3 * (3 * seg) <= cbytes
            for i in range(m):                                      # the staged pooling's reads
                assert 3 * i + 2 < n                                # z-buffer words of the item's rows
                o = (9 * i) & 3
                wb = 9 * i - o
                assert (9 * (I0 + i)) % 4 == o                      # the same byte phase as the global row
                assert 9 * i + 8 < 3 * n                            # the colour bytes used lie in the row
                assert 2 * 3 * seg + wb + 12 <= cbytes              # the three words read stay in the buffer
    if (W, H) == (1920, 1080):
        assert n_staged == 360 * 3                                  # every item of a 1080p frame is staged
