// Host-logic check of the warp-cube staging tables (make_cube_tables): for
// random gates (k = 1..6; low, high and mixed targets; 8..34 qubits) every
// 16-byte chunk a lane copies lands in two free slots, every (slice row,
// member) slot holds exactly the amplitude Eq. 3 gathers for it (slice base
// by zero insertion, Eq. 4), all addresses lie inside the state, the chunk
// accesses of each 8-lane phase hit 8 different 16-byte bank groups and the
// row accesses of each half-warp at most 2-way share a bank pair (2-way only
// when qubit 0 is a target, whose rows then move as 16-byte member pairs
// without conflicts).  Prints the counts; exit status 1 on a mismatch.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <set>
#include <vector>
#include <algorithm>
#include "internal.h"
using namespace cast;
static uint64_t slice_base(uint64_t t, const int *q, int k) {
    for (int i = 0; i < k; i++) { uint64_t low = t & ((1ull << q[i]) - 1); t = ((t >> q[i]) << (q[i] + 1)) | low; }
    return t;
}
int main() {
    srand(11);
    int bad = 0, worst_row = 0, worst_row_q0 = 0, worst_chunk = 0, worst_pair = 0;
    for (int trial = 0; trial < 30000; trial++) {
        int k = 1 + rand() % 6;
        int n = k + 7 + rand() % 20; if (n > 34) n = 34;
        int q[7]; std::set<int> s;
        int mode = trial % 3;
        if (mode == 0) for (int i = 0; i < k; i++) s.insert(i);
        else if (mode == 1) for (int i = 0; i < k; i++) s.insert(n - 1 - i);
        else while ((int)s.size() < k) s.insert(rand() % n);
        int i = 0; for (int x : s) q[i++] = x;
        CubeTables ct = make_cube_tables(q, k);
        int mb = k < 4 ? k : 4, nb = 5 + mb, rounds = (1 << nb) / 64, M = 1 << mb;
        uint64_t ncubes = 1ull << (n - k - 5);
        uint64_t c = (((uint64_t)rand() << 20) ^ rand()) % ncubes;
        int group = k > 4 ? rand() % (1 << (k - 4)) : 0;
        int j0 = 16 * group;
        uint64_t off0 = 0; for (int i2 = 4; i2 < k; i2++) if ((j0 >> i2) & 1) off0 += 1ull << q[i2];
        uint64_t wb = slice_base(c * 32, q, k) + off0;
        std::vector<uint64_t> addr(1 << nb, ~0ull);
        for (int lane = 0; lane < 32; lane++) for (int j = 0; j < rounds; j++) {
            uint32_t sl = ct.s_lane[lane] ^ ct.s_j[j];
            uint64_t g = wb + ct.g_lane[lane] + ct.g_j[j];
            if ((g & 1) || (sl & 1) || sl + 1 >= (1u << nb) + 1) bad++;
            if (sl + 1 < addr.size()) {
                if (addr[sl] != ~0ull || addr[sl + 1] != ~0ull) bad++;
                addr[sl] = g; addr[sl + 1] = g + 1;
            } else bad++;
            if ((g + 1) >> n) bad++;
        }
        for (int r = 0; r < 32; r++) for (int m = 0; m < M; m++) {
            uint32_t sl = ct.s_row[r] ^ ct.s_mem[m];
            uint64_t want = slice_base(c * 32 + r, q, k);
            int mm = j0 + m; for (int i2 = 0; i2 < k; i2++) if ((mm >> i2) & 1) want += 1ull << q[i2];
            if (sl >= addr.size() || addr[sl] != want) bad++;
        }
        for (int m = 0; m < M; m++) for (int hw = 0; hw < 2; hw++) {
            int cnt[16] = {0}, mx = 0;
            for (int r = 16 * hw; r < 16 * hw + 16; r++) { int bp = (ct.s_row[r] ^ ct.s_mem[m]) % 16; mx = std::max(mx, ++cnt[bp]); }
            if (q[0] == 0) worst_row_q0 = std::max(worst_row_q0, mx); else worst_row = std::max(worst_row, mx);
        }
        // qubit 0 a target: member pairs (2m, 2m+1) share a 16-byte chunk, in
        // order, and 16-byte row accesses (8 lanes per phase) do not conflict
        if ((ct.pair != 0) != (q[0] == 0)) bad++;
        if (ct.pair) {
            for (int r = 0; r < 32; r++) if (ct.s_row[r] & 1) bad++;
            for (int m = 0; m + 1 < M; m += 2) if (ct.s_mem[m + 1] != (ct.s_mem[m] ^ 1) || (ct.s_mem[m] & 1)) bad++;
            for (int m = 0; m < M; m += 2) for (int p = 0; p < 4; p++) {
                int cnt[8] = {0}, mx = 0;
                for (int r = 8 * p; r < 8 * p + 8; r++) { int cp = ((ct.s_row[r] ^ ct.s_mem[m]) >> 1) % 8; mx = std::max(mx, ++cnt[cp]); }
                worst_pair = std::max(worst_pair, mx);
            }
        }
        for (int j = 0; j < rounds; j++) for (int p = 0; p < 4; p++) {
            int cnt[8] = {0}, mx = 0;
            for (int lane = 8 * p; lane < 8 * p + 8; lane++) { int cp = ((ct.s_lane[lane] ^ ct.s_j[j]) >> 1) % 8; mx = std::max(mx, ++cnt[cp]); }
            worst_chunk = std::max(worst_chunk, mx);
        }
    }
    printf("bad=%d worst_row(q0!=0)=%d worst_row(q0==0)=%d worst_chunk=%d worst_pair=%d\n", bad, worst_row,
           worst_row_q0, worst_chunk, worst_pair);
    return bad != 0;
}
