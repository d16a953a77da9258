// Agglomerative, sparsity-aware gate fusion (Section IV of the paper,
// Algorithm 1 "Tile Traversal in Agglomerative Gate Fusion").
//
// CircuitTile (Section IV-A): rows of slots, one slot per qubit, each slot
// empty or naming the GateBlock that occupies that qubit in that row.  A new
// gate goes to the first row below every row that occupies one of its qubits
// (the "uppermost vacant row" that keeps the gate order on every wire).
//
// Traverse(T, k) visits rows top to bottom.  In row r, for each qubit q with a
// block b_top:
//   - if every slot of b_top's qubits in row r+1 is empty, b_top moves down to
//     row r+1 (MoveBlock; it is visited again there);
//   - otherwise b_bot = T[r+1][q]; if Fusible(b_top, b_bot, k) they are fused
//     (consecutive fusion, product U_bot * U_top).
// Then for q = 1..n-1 the horizontally adjacent blocks T[r][q-1], T[r][q] are
// fused if Fusible (commuting fusion of disjoint blocks).
// Fuse removes both blocks and places the product in row r+1 if all its slots
// there are free, else in row r, else in a new row inserted between r and
// r+1.  Empty rows are removed after each traversal (compression).
//
// Fusible: distinct non-empty blocks whose qubit union has at most k qubits;
// adaptive mode adds the cost-model test of Section IV-C: the fused operation
// count (2 per non-zero real scalar) is at most op_cap and the fused block's
// estimated time is not above the two blocks' sum.  The estimate of a block
// with k qubits and operation count ops, per amplitude of the state and in
// integer units, is max(P * 128, ops * 2^(7-k)) with P the operation count per
// amplitude that costs as much as one pass over memory.
//
// Agglomerative schedule (Section IV-B): the allowed size grows 2, 3, ...,
// max_k; at each size Traverse repeats until it fuses nothing.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include <utility>

#include "internal.h"

namespace cast {

namespace {

struct Block {
    std::vector<int> q;   // sorted ascending
    std::vector<cplx> m;  // 4^k row-major over q
    int64_t ops = 0;
};

struct Tile {
    int nq;
    std::vector<std::vector<int>> rows;  // rows[r][q] = block id or -1
};

// Offsets of the 2^k member indices of a gate on positions pos (bit i of j
// sets bit pos[i]).
std::vector<size_t> member_offsets(const std::vector<int> &pos) {
    const size_t dk = size_t(1) << pos.size();
    std::vector<size_t> off(dk, 0);
    for (size_t j = 0; j < dk; j++)
        for (size_t i = 0; i < pos.size(); i++)
            if ((j >> i) & 1) off[j] |= size_t(1) << pos[i];
    return off;
}

// M <- lift(U on positions pos) * M; M is ku-qubit (2^ku x 2^ku).  The rows
// of M fall into groups of 2^k that differ only at pos; each group is
// replaced by U times it, whole rows at a time (contiguous in memory).  Every
// output entry sums its products in the order of U's columns, skipping zero
// entries of U (their products add nothing).
void left_apply(std::vector<cplx> &M, int ku, const std::vector<cplx> &U, const std::vector<int> &pos) {
    const size_t du = size_t(1) << ku, dk = size_t(1) << pos.size();
    const std::vector<size_t> off = member_offsets(pos);
    const size_t tmask = off[dk - 1];
    std::vector<cplx> rows(dk * du);
    for (size_t b = 0; b < du; b++) {
        if (b & tmask) continue;
        for (size_t j = 0; j < dk; j++) std::copy_n(&M[(b + off[j]) * du], du, &rows[j * du]);
        for (size_t r = 0; r < dk; r++) {
            cplx *out = &M[(b + off[r]) * du];
            std::fill_n(out, du, cplx(0.0, 0.0));
            for (size_t c = 0; c < dk; c++) {
                const cplx u = U[r * dk + c];
                if (u == cplx(0.0, 0.0)) continue;
                const cplx *x = &rows[c * du];
                for (size_t col = 0; col < du; col++) out[col] += u * x[col];
            }
        }
    }
}

// M <- M * lift(U on positions pos), the same way by columns: in every row,
// the 2^k entries that differ only at pos are replaced by their product
// with U (sums in the order of U's rows, zero entries skipped).
void right_apply(std::vector<cplx> &M, int ku, const std::vector<cplx> &U, const std::vector<int> &pos) {
    const size_t du = size_t(1) << ku, dk = size_t(1) << pos.size();
    const std::vector<size_t> off = member_offsets(pos);
    const size_t tmask = off[dk - 1];
    std::vector<cplx> x(dk), y(dk);
    for (size_t r = 0; r < du; r++) {
        cplx *row = &M[r * du];
        for (size_t b = 0; b < du; b++) {
            if (b & tmask) continue;
            for (size_t c = 0; c < dk; c++) x[c] = row[b + off[c]];
            std::fill(y.begin(), y.end(), cplx(0.0, 0.0));
            for (size_t c = 0; c < dk; c++) {
                if (x[c] == cplx(0.0, 0.0)) continue;
                const cplx *u = &U[c * dk];
                for (size_t j = 0; j < dk; j++)
                    if (u[j] != cplx(0.0, 0.0)) y[j] += x[c] * u[j];
            }
            for (size_t j = 0; j < dk; j++) row[b + off[j]] = y[j];
        }
    }
}

// lift(U on positions pos) as a ku-qubit matrix: entry (r, c) is U's entry of
// their member bits where r and c agree at every other position, else 0
std::vector<cplx> lift(int ku, const std::vector<cplx> &U, const std::vector<int> &pos) {
    const size_t du = size_t(1) << ku;
    std::vector<cplx> M(du * du, cplx(0.0, 0.0));
    const std::vector<size_t> off = member_offsets(pos);
    const size_t dk = off.size(), mask = off[dk - 1];
    for (size_t b = 0; b < du; b++) {
        if (b & mask) continue;
        for (size_t r = 0; r < dk; r++)
            for (size_t c = 0; c < dk; c++) M[(b + off[r]) * du + b + off[c]] = U[r * dk + c];
    }
    return M;
}

std::vector<int> union_q(const Block &a, const Block &b) {
    std::vector<int> u;
    std::set_union(a.q.begin(), a.q.end(), b.q.begin(), b.q.end(), std::back_inserter(u));
    return u;
}

std::vector<int> positions(const std::vector<int> &sub, const std::vector<int> &all) {
    std::vector<int> p;
    for (int q : sub) p.push_back(int(std::lower_bound(all.begin(), all.end(), q) - all.begin()));
    return p;
}

// Product "second after first" on the union of their qubits.
Block product(const Block &first, const Block &second, double tol) {
    Block f;
    f.q = union_q(first, second);
    const int ku = (int)f.q.size();
    // second * first on the union: lift the larger block and apply the
    // smaller one to it (2^(2 ku) times the smaller dimension operations)
    if (second.q.size() <= first.q.size()) {
        f.m = lift(ku, first.m, positions(first.q, f.q));
        left_apply(f.m, ku, second.m, positions(second.q, f.q));
    } else {
        f.m = lift(ku, second.m, positions(second.q, f.q));
        right_apply(f.m, ku, first.m, positions(first.q, f.q));
    }
    f.ops = opcount(f.m.data(), ku, tol);
    return f;
}

struct Fuser {
    const cast_options &opt;
    int64_t P;  // operation count per amplitude equal to one memory pass
    std::vector<Block> blocks;
    std::vector<char> alive;
    Tile T;
    // pairs (first, second) the cost test refused: blocks never change (a
    // fusion makes a new block), and the test does not depend on the size
    // limit, so a later traversal refuses them again without the product
    std::set<std::pair<int, int>> refused;

    int64_t cost(const Block &b) const {
        const int k = (int)b.q.size();
        if (opt.cost) return table_estimate(*opt.cost, k, classify_matrix(b.m.data(), k, opt.zero_tol), b.ops);
        const int64_t mem = P * 128;
        const int64_t cmp = b.ops << (7 - k);
        return mem > cmp ? mem : cmp;
    }

    bool row_free(int r, const std::vector<int> &qs) const {
        if (r < 0 || r >= (int)T.rows.size()) return false;
        for (int q : qs)
            if (T.rows[r][q] >= 0) return false;
        return true;
    }
    void place(int r, int id) {
        for (int q : blocks[id].q) T.rows[r][q] = id;
    }
    void remove(int r, int id) {
        for (int q : blocks[id].q)
            if (T.rows[r][q] == id) T.rows[r][q] = -1;
    }

    void append(Block b) {
        const int id = (int)blocks.size();
        blocks.push_back(std::move(b));
        alive.push_back(1);
        int last = -1;
        for (int r = (int)T.rows.size() - 1; r >= 0 && last < 0; r--)
            for (int q : blocks[id].q)
                if (T.rows[r][q] >= 0) { last = r; break; }
        const int r = last + 1;
        if (r == (int)T.rows.size()) T.rows.emplace_back(T.nq, -1);
        place(r, id);
    }

    // size + (adaptive) cost test; on success the product is returned in *out
    bool fusible(int top, int bot, int k, bool consecutive, Block *out) {
        if (top < 0 || bot < 0 || top == bot) return false;
        const Block &a = blocks[top], &b = blocks[bot];
        if ((int)union_q(a, b).size() > k) return false;
        // consecutive: a (upper row) acts first; commuting: disjoint, any order
        (void)consecutive;
        const bool adaptive = opt.fusion == CAST_FUSE_ADAPTIVE;
        if (adaptive && refused.count({top, bot})) return false;
        *out = product(a, b, opt.zero_tol);
        if (adaptive && (out->ops > opt.op_cap || cost(*out) > cost(a) + cost(b))) {
            refused.insert({top, bot});
            return false;
        }
        return true;
    }

    // remove both, place the product in r+1, else r, else a new row between
    void fuse(int r_top, int top, int r_bot, int bot, Block fused) {
        remove(r_top, top);
        remove(r_bot, bot);
        alive[top] = alive[bot] = 0;
        const int id = (int)blocks.size();
        blocks.push_back(std::move(fused));
        alive.push_back(1);
        const std::vector<int> &qs = blocks[id].q;
        const int r = r_top;  // the two rows involved are r_top and r_top + 1 (consecutive) or r_top (commuting)
        if (row_free(r + 1, qs)) {
            place(r + 1, id);
        } else if (row_free(r, qs)) {
            place(r, id);
        } else {
            T.rows.insert(T.rows.begin() + r + 1, std::vector<int>(T.nq, -1));
            place(r + 1, id);
        }
    }

    bool traverse(int k) {
        bool delta = false;
        for (int r = 0; r < (int)T.rows.size(); r++) {
            for (int q = 0; q < T.nq; q++) {
                const int top = T.rows[r][q];
                if (top < 0) continue;
                if (r + 1 < (int)T.rows.size() && row_free(r + 1, blocks[top].q)) {
                    remove(r, top);  // MoveBlock
                    place(r + 1, top);
                    continue;
                }
                if (r + 1 >= (int)T.rows.size()) continue;
                const int bot = T.rows[r + 1][q];
                Block f;
                if (fusible(top, bot, k, true, &f)) {
                    fuse(r, top, r + 1, bot, std::move(f));
                    delta = true;
                }
            }
            for (int q = 1; q < T.nq; q++) {
                const int a = T.rows[r][q - 1], b = T.rows[r][q];
                Block f;
                if (fusible(a, b, k, false, &f)) {
                    fuse(r, a, r, b, std::move(f));
                    delta = true;
                }
            }
        }
        return delta;
    }

    void compress() {
        std::vector<std::vector<int>> kept;
        for (auto &row : T.rows) {
            bool any = false;
            for (int v : row) any |= v >= 0;
            if (any) kept.push_back(std::move(row));
        }
        T.rows.swap(kept);
    }

    // one size of the schedule: traverse until nothing fuses
    void grow(int k) {
        while (traverse(k)) compress();
        compress();
    }

    void run() {
        if (opt.fusion == CAST_FUSE_NONE) return;
        const int kmax = opt.max_k;
        const int k0 = opt.agglomerative ? std::min(2, kmax) : kmax;
        for (int k = k0; k <= kmax; k++) grow(k);
    }
};

}  // namespace

// Operations per amplitude that take as long as one pass over the state:
// complex64 FP32 FMA 82; complex128 on the FP64 pipe 2 (measured rates on
// GB300).  complex128 in the emulated mode runs dense gates of k >= 4 on the
// tensor cores (digit products) and sparse ones on the list kernel: measured
// on a random 30-qubit state, every gate of k <= 5 costs 1.5 to 6.3 passes
// (7.7 ms diagonal, 13.2 ms dense k = 2, 24 ms dense k = 3, 4, 32 ms dense
// k = 5) with no slope in the operation count the model could follow, and
// merging pays almost always; 64 puts every gate of k <= 5 on the floor
// P * 128, which reproduces the plans the measured cost table picks on the
// six benchmark families (the 16 of the double-float CUDA-core kernels fused
// too little: up to 1.6x slower than size-only).
int64_t default_amp_ops_per_pass(cast_dtype dt) {
    if (dt == CAST_C64) return 82;
    return f64_mode() == CAST_F64_EMULATED ? 64 : 2;
}

namespace {

// The circuit's gates as the first blocks of F, in order.
cast_status load_circuit(const cast_circuit *c, const double *params, const cast_options *opt, Fuser &F) {
    for (int g = 0; g < c->n_gates; g++) {
        const cast_gate &gt = c->gates[g];
        std::vector<cplx> m;
        cast_status st = gate_matrix_of(gt, params, c->n_params, &m);
        if (st != CAST_OK) return st;
        PreparedGate pg;
        st = prepare_gate(c->n_qubits, gt.qubits, gt.k, m.data(), opt->zero_tol, &pg);
        if (st != CAST_OK) return st;
        Block b;
        b.q.assign(pg.q, pg.q + pg.k);
        b.m = pg.m;
        b.ops = opcount(b.m.data(), pg.k, opt->zero_tol);
        F.append(std::move(b));
    }
    return CAST_OK;
}

// The current blocks in plan order: rows top to bottom, each row by qubit.
void emit(const Fuser &F, std::vector<FusedGate> *out) {
    out->clear();
    std::vector<char> emitted(F.blocks.size(), 0);
    for (auto &row : F.T.rows)
        for (int q = 0; q < F.T.nq; q++) {
            const int id = row[q];
            if (id < 0 || emitted[id]) continue;
            emitted[id] = 1;
            FusedGate fg;
            const Block &b = F.blocks[id];
            fg.k = (int)b.q.size();
            for (int i = 0; i < CAST_MAX_K; i++) fg.q[i] = i < fg.k ? b.q[i] : -1;
            fg.m = b.m;
            fg.ops = b.ops;
            out->push_back(std::move(fg));
        }
}

int64_t amp_ops_per_pass(const cast_options *opt) {
    return opt->amp_ops_per_pass > 0 ? opt->amp_ops_per_pass : default_amp_ops_per_pass(CAST_C64);
}

}  // namespace

// With a cost table and max_k = 0, try every fusion width and keep the plan of
// least estimated time (ties: the smaller width).  The agglomerative
// schedule of width w is that of width w - 1 followed by one more size, so
// one schedule grown to the largest width yields every candidate plan.
cast_status fuse_circuit(const cast_circuit *c, const double *params, const cast_options *opt,
                         std::vector<FusedGate> *out) {
    const bool search = opt->cost && opt->max_k == 0;
    if (!search || !opt->agglomerative || opt->fusion == CAST_FUSE_NONE) {
        int64_t best = -1;
        for (int k = search ? 2 : opt->max_k; k <= (search ? CAST_MAX_K : opt->max_k); k++) {
            cast_options o = *opt;
            o.max_k = k;
            Fuser F{o, amp_ops_per_pass(opt), {}, {}, {c->n_qubits, {}}};
            cast_status st = load_circuit(c, params, opt, F);
            if (st != CAST_OK) return st;
            F.run();
            std::vector<FusedGate> cand;
            emit(F, &cand);
            if (!search) {
                out->swap(cand);
                return CAST_OK;
            }
            int64_t total = 0;
            for (const FusedGate &g : cand)
                total += table_estimate(*opt->cost, g.k, classify_matrix(g.m.data(), g.k, o.zero_tol), g.ops);
            if (best < 0 || total < best) {
                best = total;
                out->swap(cand);
            }
        }
        return CAST_OK;
    }
    cast_options o = *opt;
    o.max_k = CAST_MAX_K;
    Fuser F{o, amp_ops_per_pass(opt), {}, {}, {c->n_qubits, {}}};
    cast_status st = load_circuit(c, params, opt, F);
    if (st != CAST_OK) return st;
    int64_t best = -1;
    for (int k = 2; k <= CAST_MAX_K; k++) {
        F.grow(k);
        std::vector<FusedGate> cand;
        emit(F, &cand);
        int64_t total = 0;
        for (const FusedGate &g : cand)
            total += table_estimate(*opt->cost, g.k, classify_matrix(g.m.data(), g.k, o.zero_tol), g.ops);
        if (best < 0 || total < best) {
            best = total;
            out->swap(cand);
        }
    }
    return CAST_OK;
}

}  // namespace cast
