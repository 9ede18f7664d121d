"""Index arithmetic of the shared-memory exchange layouts, checked on the CPU (no GPU needed): for every pencil
length, radix and tile width the kernels can use, the column-tile layout's row permutation is a bijection onto
the buffer and the padded row layout stays inside its buffer.  The formulas restate csrc/fft.cuh."""
import pytest


def col_idx(p, c, N, TC, E, elem_bytes):
    per_phase = 128 // elem_bytes
    g0 = per_phase // TC
    g1 = 1 if g0 < 1 else g0
    g = E if g1 > E else g1
    q = p if g == 1 else (p & ~(g - 1)) + ((p + p // E) & (g - 1))
    return q * TC + c


@pytest.mark.parametrize("elem_bytes", [8, 16])
def test_column_layout_is_a_bijection(elem_bytes):
    for N in (8, 16, 32, 64, 128, 256, 512):
        for E in (4, 8, 16, 32):
            if E > N:
                continue
            for TC in (1, 2, 4, 8, 16, 32, 64, 128):
                got = {col_idx(p, c, N, TC, E, elem_bytes) for p in range(N) for c in range(TC)}
                assert got == set(range(N * TC)), (N, TC, E, elem_bytes)


@pytest.mark.parametrize("padsh", [3, 4, 5])
def test_row_layout_fits_its_buffer(padsh):
    for N in (8, 16, 32, 64, 128, 256, 512):
        buf = N + (N - 1) // (1 << padsh) + 1
        idx = [p + (p >> padsh) for p in range(N)]
        assert len(set(idx)) == N and max(idx) < buf
