// Host-logic check of the list kernel's super-tile mapping (make_tile_layout
// and the index arithmetic of k_sparse in apply_sparse.cu, restated here):
// for random gates (k = 3..7; low, high and mixed targets; 12..34 qubits) the
// 256 threads x 16 elements of a super-tile address 4096 distinct amplitudes,
// each exactly the one Eq. 3 gathers for its (slice row, member) -- slice
// base by zero insertion (Eq. 4) plus the member's target bits -- and 4096
// distinct shared-memory slots inside the [G][D][33] buffer; a thread's slot
// and address are the sums of its cube bits 0..7 part and the element's bits
// 8..11 part (the per-CTA table form).  Prints the counts; exit status 1 on
// a mismatch.
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
    srand(17);
    const int SP = 33;
    int bad = 0, gates = 0;
    for (int trial = 0; trial < 3000; trial++) {
        const int k = 3 + rand() % 5, D = 1 << k, G = 1 << (7 - k);
        int n = 12 + rand() % 23; if (n < k + 5) n = k + 5;
        int q[7]; std::set<int> s;
        const int mode = trial % 3;
        if (mode == 0) for (int i = 0; i < k; i++) s.insert(i);
        else if (mode == 1) for (int i = 0; i < k; i++) s.insert(n - 1 - i);
        else while ((int)s.size() < k) s.insert(rand() % n);
        int i0 = 0; for (int v : s) q[i0++] = v;
        const SpTile lay = make_tile_layout(q, k);
        const uint64_t nsuper = uint64_t(1) << (n - 12);
        const uint64_t sts[3] = {0, nsuper - 1, uint64_t(rand()) % nsuper};
        // the per-element part (cube bits 8..11), as the kernel's table holds it
        uint64_t aU[16]; uint32_t sU[16], slU[16], jU[16];
        for (int u = 0; u < 16; u++) {
            uint64_t a = 0; uint32_t ss = 0, j = 0;
            for (int b = 8; b < 12; b++) {
                if (!((u >> (b - 8)) & 1)) continue;
                a += uint64_t(1) << lay.pos[b];
                const int r = lay.role[b];
                if (r < 16) ss |= 1u << r; else j |= 1u << (r - 16);
            }
            aU[u] = a; sU[u] = ss; jU[u] = j;
            slU[u] = ((ss >> 5) * D + j) * SP + (ss & 31);
        }
        for (uint64_t st : sts) {
            const uint64_t base = slice_base(st * (32 * G), q, k);
            std::set<uint64_t> addrs; std::set<uint32_t> slots;
            for (int tid = 0; tid < 256; tid++) {
                uint64_t alo = 0; uint32_t slo = 0, jlo = 0;
                for (int b = 0; b < 8; b++) {
                    if (!((tid >> b) & 1)) continue;
                    alo += uint64_t(1) << lay.pos[b];
                    const int r = lay.role[b];
                    if (r < 16) slo |= 1u << r; else jlo |= 1u << (r - 16);
                }
                const uint32_t sl_lo = ((slo >> 5) * D + jlo) * SP + (slo & 31);
                for (int u = 0; u < 16; u++) {
                    const uint64_t a = base + alo + aU[u];
                    const uint32_t srow = slo | sU[u], j = jlo | jU[u];
                    const uint32_t slot = sl_lo + slU[u];
                    // the table form equals the slot of the whole (row, member)
                    if (slot != ((srow >> 5) * D + j) * SP + (srow & 31)) bad++;
                    if ((slo & sU[u]) || (jlo & jU[u])) bad++;
                    if (srow >= uint32_t(32 * G) || j >= uint32_t(D) || slot >= uint32_t(G * D * SP)) bad++;
                    // Eq. 3: member j of slice st * 32G + srow
                    uint64_t want = slice_base(st * (32 * G) + srow, q, k);
                    for (int i = 0; i < k; i++) if ((j >> i) & 1) want += uint64_t(1) << q[i];
                    if (a != want || a >= (uint64_t(1) << n)) bad++;
                    addrs.insert(a); slots.insert(slot);
                }
            }
            if (addrs.size() != 4096 || slots.size() != 4096) bad++;
            gates++;
        }
    }
    printf("checked=%d bad=%d\n", gates, bad);
    return bad ? 1 : 0;
}
