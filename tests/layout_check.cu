// Host-only checks of the neighbour-data layout helpers of d3gb_internal.cuh
// (no kernel is launched; compiled and run by tests/test_layout_host.py):
//  * per-atom list rows interleaved across 32 atoms: every (atom, entry) maps to
//    a distinct slot inside the structure's list_size, groups of 4 entries start
//    on 16-byte boundaries, and the 32 atoms of a group read entries 4m..4m+3 as
//    one contiguous run of 128 slots;
//  * serpentine cell numbering: cell_index and cell_coords are inverse over every
//    cell, consecutive ids are face neighbours, and row_cells spans exactly the
//    cells of a row between two x bounds.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_2310_05279_gb300/csrc/d3gb_internal.cuh"

using namespace d3gb;

static int failures = 0;
#define CHECK(cond, ...)                     \
    do {                                     \
        if (!(cond)) {                       \
            if (failures < 20) {             \
                std::printf("FAIL: ");       \
                std::printf(__VA_ARGS__);    \
                std::printf("\n");           \
            }                                \
            ++failures;                      \
        }                                    \
    } while (0)

static void check_lists(int64_t natoms, int cap, int64_t base) {
    const int64_t size = list_size(natoms, cap);
    CHECK(size >= natoms * cap, "list_size(%lld, %d) too small", (long long)natoms, cap);
    std::vector<char> seen((size_t)size, 0);
    for (int64_t a = 0; a < natoms; ++a) {
        const int64_t row = list_row(base, a, cap);
        CHECK(row % 4 == 0, "row of atom %lld not 16-byte aligned", (long long)a);
        for (int k = 0; k < cap; ++k) {
            const int64_t s = row + list_off(k) - base;
            CHECK(s >= 0 && s < size, "slot out of range: atom %lld entry %d", (long long)a, k);
            if (s < 0 || s >= size) continue;
            CHECK(!seen[(size_t)s], "slot used twice: atom %lld entry %d", (long long)a, k);
            seen[(size_t)s] = 1;
            if (k % 4 == 0) CHECK((row + list_off(k)) % 4 == 0, "group not aligned: atom %lld entry %d", (long long)a, k);
            if (k % 4 != 0) CHECK(list_off(k) == list_off(k - 1) + 1, "group not contiguous at entry %d", k);
        }
    }
    // a full group of 32 atoms reads entries 4m..4m+3 as one run of 128 slots
    for (int64_t g = 0; (g + 1) * 32 <= natoms; ++g)
        for (int m = 0; m < cap / 4; ++m) {
            const int64_t first = list_row(base, 32 * g, cap) + list_off(4 * m);
            for (int l = 0; l < 32; ++l)
                CHECK(list_row(base, 32 * g + l, cap) + list_off(4 * m) == first + 4 * l,
                      "warp read not contiguous: group %lld entries %d", (long long)g, 4 * m);
        }
}

static void check_cells(int nx, int ny, int nz, int64_t cell_base) {
    StructGeo G{};
    G.ncell[0] = nx;
    G.ncell[1] = ny;
    G.ncell[2] = nz;
    G.cell_base = cell_base;
    const int64_t n = (int64_t)nx * ny * nz;
    std::vector<char> seen((size_t)n, 0);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int64_t id = cell_index(G, x, y, z);
                CHECK(id >= cell_base && id < cell_base + n, "cell id out of range");
                if (id < cell_base || id >= cell_base + n) continue;
                CHECK(!seen[(size_t)(id - cell_base)], "cell id used twice");
                seen[(size_t)(id - cell_base)] = 1;
                int cx, cy, cz;
                cell_coords(G, id, cx, cy, cz);
                CHECK(cx == x && cy == y && cz == z, "cell_coords does not invert cell_index at (%d, %d, %d)", x, y, z);
            }
    // consecutive ids are face neighbours (the serpentine property)
    for (int64_t id = cell_base; id + 1 < cell_base + n; ++id) {
        int ax, ay, az, bx, by, bz;
        cell_coords(G, id, ax, ay, az);
        cell_coords(G, id + 1, bx, by, bz);
        const int d = std::abs(ax - bx) + std::abs(ay - by) + std::abs(az - bz);
        CHECK(d == 1, "cells %lld and %lld are not face neighbours", (long long)id, (long long)id + 1);
    }
    // row_cells: the ids between first and last are exactly the cells x0..x1 of the row
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x0 = 0; x0 < nx; ++x0)
                for (int x1 = x0; x1 < nx; ++x1) {
                    int64_t first, last;
                    row_cells(G, y, z, x0, x1, first, last);
                    CHECK(last - first == x1 - x0, "row_cells span wrong");
                    for (int64_t id = first; id <= last; ++id) {
                        int cx, cy, cz;
                        cell_coords(G, id, cx, cy, cz);
                        CHECK(cy == y && cz == z && cx >= x0 && cx <= x1, "row_cells holds a cell outside the row");
                    }
                }
}

int main() {
    const int64_t natoms[] = {1, 7, 31, 32, 33, 64, 100, 1440};
    const int caps[] = {8, 16, 24, 64};
    for (int64_t n : natoms)
        for (int cap : caps) check_lists(n, cap, 256);
    const int dims[][3] = {{1, 1, 1}, {3, 4, 5}, {7, 2, 3}, {2, 5, 1}, {4, 4, 4}, {1, 6, 2}};
    for (const auto& d : dims) {
        check_cells(d[0], d[1], d[2], 0);
        check_cells(d[0], d[1], d[2], 17);
    }
    if (failures) {
        std::printf("%d failures\n", failures);
        return 1;
    }
    std::printf("OK\n");
    return 0;
}
