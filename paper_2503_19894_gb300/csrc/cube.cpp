// Host-built staging tables of a warp's cube (struct CubeTables in
// internal.h): the gather of Eq. 3 for 32 consecutive slices, laid out so that
// the warp moves it between HBM and shared memory with coalesced 16-byte
// chunks and every lane then reads its own slice row.  Also the bit layout of
// the list kernel's 4096-amplitude super-tiles (struct SpTile).
#include "internal.h"

namespace cast {

// For sorted targets q[0..k): the cube's 5 + mb address bits are the 5 lowest
// non-target bits (row bits r0..r4) and q0..q_{mb-1} (member bits), mb =
// min(k, 4), in ascending order; cube position b holds address bit abit[b].
// Address bits 0..4 are always among them (each is either a target among
// the lowest ones or one of the 5 lowest non-targets).  The swizzle X sends
// each of r0..r3 at a position >= 4 to a free slot bit among 1..3, so that
// the 16 rows of a half-warp land in different 8-byte bank pairs (when
// qubit 0 is a target only three slot bits are free: 2-way at most).
CubeTables make_cube_tables(const int *q, int k) { return make_cube_tables(q, k, k < 4 ? k : 4); }

CubeTables make_cube_tables(const int *q, int k, int mb) {
    const int nbits = 5 + mb;
    int rpos[5], mpos[4] = {0, 0, 0, 0}, abit[9];
    int nr = 0, nm = 0, nb = 0;
    for (int a = 0; nb < nbits; a++) {
        int ti = -1;
        for (int i = 0; i < k; i++)
            if (q[i] == a) ti = i;
        if (ti >= 0 && ti < mb) {
            mpos[nm++] = nb;
            abit[nb++] = a;
        } else if (ti < 0 && nr < 5) {
            rpos[nr++] = nb;
            abit[nb++] = a;
        }
    }
    uint32_t contrib[9] = {0};
    uint32_t used = 1u;  // slot bit 0 stays: a 16-byte chunk keeps its two amplitudes in order
    for (int h = 0; h < 4; h++)
        if (rpos[h] < 4) used |= 1u << rpos[h];
    int next_free = 1;
    for (int h = 0; h < 4; h++)
        if (rpos[h] >= 4) {
            while (next_free < 4 && (used & (1u << next_free))) next_free++;
            if (next_free >= 4) break;
            contrib[rpos[h]] = 1u << next_free;
            used |= 1u << next_free;
        }
    auto slot = [&](uint32_t c) {
        uint32_t x = c;
        for (int b = 4; b < nbits; b++)
            if ((c >> b) & 1) x ^= contrib[b];
        return uint16_t(x);
    };
    auto goff = [&](uint32_t c) {
        uint64_t o = 0;
        for (int b = 0; b < nbits; b++)
            if ((c >> b) & 1) o += uint64_t(1) << abit[b];
        return o;
    };
    auto deposit = [&](uint32_t v, const int *pos, int cnt) {
        uint32_t c = 0;
        for (int i = 0; i < cnt; i++)
            if ((v >> i) & 1) c |= 1u << pos[i];
        return c;
    };
    CubeTables ct{};
    for (int i = 0; i < 32; i++) {
        ct.g_lane[i] = goff(2u * i);
        ct.s_lane[i] = slot(2u * i);
        ct.s_row[i] = slot(deposit(uint32_t(i), rpos, 5));
    }
    const int rounds = (1 << nbits) / 64;  // chunks of 2 amplitudes per lane
    for (int j = 0; j < 8; j++) {
        ct.g_j[j] = j < rounds ? goff(64u * j) : 0;
        ct.s_j[j] = j < rounds ? slot(64u * j) : 0;
    }
    for (int m = 0; m < 16; m++) ct.s_mem[m] = m < (1 << mb) ? slot(deposit(uint32_t(m), mpos, mb)) : 0;
    ct.pair = (k >= 1 && q[0] == 0) ? 1u : 0u;
    return ct;
}

SpTile make_tile_layout(const int *q, int k) {
    // 12 cube bits: the 12 - k lowest non-target positions (slice row bits)
    // and the k targets, ascending
    SpTile t{};
    int nb = 0, nr = 0;
    for (int a = 0; nb < 12; a++) {
        int ti = -1;
        for (int i = 0; i < k; i++)
            if (q[i] == a) ti = i;
        if (ti >= 0) {
            t.pos[nb] = (uint8_t)a;
            t.role[nb++] = (uint8_t)(16 + ti);
        } else if (nr < 12 - k) {
            t.pos[nb] = (uint8_t)a;
            t.role[nb++] = (uint8_t)nr++;
        }
    }
    return t;
}

}  // namespace cast
