// Gate table, gate preparation (validate, sort qubits, snap zeros, classify)
// and the operation count of Section IV-C.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace cast {

namespace {
const double kInvSqrt2 = 0.70710678118654752440;
}

int gate_table_arity(int kind) {
    switch (kind) {
        case CAST_GATE_H: case CAST_GATE_X: case CAST_GATE_Y: case CAST_GATE_Z:
        case CAST_GATE_S: case CAST_GATE_T: case CAST_GATE_RX: case CAST_GATE_RY:
        case CAST_GATE_RZ: case CAST_GATE_U3:
            return 1;
        case CAST_GATE_CX: case CAST_GATE_CZ: case CAST_GATE_CP: case CAST_GATE_SWAP:
            return 2;
        default:
            return 0;
    }
}

// Row-major 2^k x 2^k matrices.  Local bit i <-> the gate's i-th qubit; for
// the controlled gates bit 0 is the control.
cast_status gate_table_matrix(int kind, int k, const double *p, std::vector<cplx> *out) {
    const int ar = gate_table_arity(kind);
    if (ar == 0 || ar != k) return fail(CAST_ERR_ARG, "gate kind/arity mismatch");
    const cplx I(0.0, 1.0);
    std::vector<cplx> &m = *out;
    m.assign(size_t(1) << (2 * k), cplx(0.0, 0.0));
    auto at = [&](int r, int c) -> cplx & { return m[size_t(r) * (size_t(1) << k) + c]; };
    switch (kind) {
        case CAST_GATE_H:
            at(0, 0) = at(0, 1) = at(1, 0) = kInvSqrt2;
            at(1, 1) = -kInvSqrt2;
            break;
        case CAST_GATE_X: at(0, 1) = at(1, 0) = 1.0; break;
        case CAST_GATE_Y: at(0, 1) = -I; at(1, 0) = I; break;
        case CAST_GATE_Z: at(0, 0) = 1.0; at(1, 1) = -1.0; break;
        case CAST_GATE_S: at(0, 0) = 1.0; at(1, 1) = I; break;
        case CAST_GATE_T: at(0, 0) = 1.0; at(1, 1) = std::polar(1.0, M_PI / 4); break;
        case CAST_GATE_RX: {  // exp(-i t X / 2) = cos(t/2) I - i sin(t/2) X
            double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
            at(0, 0) = at(1, 1) = c;
            at(0, 1) = at(1, 0) = cplx(0.0, -s);
            break;
        }
        case CAST_GATE_RY: {  // exp(-i t Y / 2)
            double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
            at(0, 0) = at(1, 1) = c;
            at(0, 1) = -s;
            at(1, 0) = s;
            break;
        }
        case CAST_GATE_RZ:  // exp(-i t Z / 2)
            at(0, 0) = std::polar(1.0, -p[0] / 2);
            at(1, 1) = std::polar(1.0, p[0] / 2);
            break;
        case CAST_GATE_U3: {
            double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
            at(0, 0) = c;
            at(0, 1) = -std::polar(s, p[2]);
            at(1, 0) = std::polar(s, p[1]);
            at(1, 1) = std::polar(c, p[1] + p[2]);
            break;
        }
        case CAST_GATE_CX:  // control = local bit 0: |01> <-> |11>
            at(0, 0) = at(2, 2) = 1.0;
            at(1, 3) = at(3, 1) = 1.0;
            break;
        case CAST_GATE_CZ:
            at(0, 0) = at(1, 1) = at(2, 2) = 1.0;
            at(3, 3) = -1.0;
            break;
        case CAST_GATE_CP:
            at(0, 0) = at(1, 1) = at(2, 2) = 1.0;
            at(3, 3) = std::polar(1.0, p[0]);
            break;
        case CAST_GATE_SWAP:
            at(0, 0) = at(3, 3) = 1.0;
            at(1, 2) = at(2, 1) = 1.0;
            break;
        default:
            return fail(CAST_ERR_ARG, "unknown gate kind");
    }
    return CAST_OK;
}

cast_status gate_matrix_of(const cast_gate &g, const double *params, int n_params,
                           std::vector<cplx> *out) {
    if (g.k < 1 || g.k > CAST_MAX_K) return fail(CAST_ERR_ARG, "gate size k must be in 1..7");
    if (g.kind == CAST_GATE_MATRIX) {
        if (!g.matrix) return fail(CAST_ERR_ARG, "explicit-matrix gate without a matrix");
        const size_t n = size_t(1) << (2 * g.k);
        out->resize(n);
        for (size_t i = 0; i < n; i++) (*out)[i] = cplx(g.matrix[2 * i], g.matrix[2 * i + 1]);
        return CAST_OK;
    }
    double p[3] = {g.params[0], g.params[1], g.params[2]};
    if (g.param_index >= 0) {
        if (g.kind != CAST_GATE_RX && g.kind != CAST_GATE_RY && g.kind != CAST_GATE_RZ &&
            g.kind != CAST_GATE_CP)
            return fail(CAST_ERR_ARG, "only RX, RY, RZ and CP gates can be parametrised");
        if (!params || g.param_index >= n_params)
            return fail(CAST_ERR_ARG, "param_index outside the parameter array");
        p[0] = params[g.param_index];
    }
    return gate_table_matrix(g.kind, g.k, p, out);
}

int classify_matrix(const cplx *m, int k, double tol) {
    const int d = 1 << k;
    auto nz = [&](int r, int c) {
        const cplx v = m[size_t(r) * d + c];
        return std::fabs(v.real()) > tol || std::fabs(v.imag()) > tol;
    };
    bool diag = true, ident = true;
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) {
            if (r != c && nz(r, c)) diag = false;
            if (r == c && std::abs(m[size_t(r) * d + c] - cplx(1.0, 0.0)) > tol) ident = false;
        }
    if (diag) return ident ? CLS_IDENTITY : CLS_DIAG;
    for (int r = 0; r < d; r++) {
        int cnt = 0;
        for (int c = 0; c < d; c++) cnt += nz(r, c);
        if (cnt != 1) return CLS_DENSE;
    }
    for (int c = 0; c < d; c++) {
        int cnt = 0;
        for (int r = 0; r < d; r++) cnt += nz(r, c);
        if (cnt != 1) return CLS_DENSE;
    }
    return CLS_MONO;
}

int64_t opcount(const cplx *m, int k, double tol) {
    const size_t n = size_t(1) << (2 * k);
    int64_t nz = 0;
    for (size_t i = 0; i < n; i++) {
        nz += std::fabs(m[i].real()) > tol;
        nz += std::fabs(m[i].imag()) > tol;
    }
    return 2 * nz;
}

cast_status prepare_gate(int n, const int *qubits, int k, const cplx *matrix, double tol,
                         PreparedGate *g) {
    if (k < 1 || k > CAST_MAX_K) return fail(CAST_ERR_ARG, "gate size k must be in 1..7");
    if (k > n) return fail(CAST_ERR_ARG, "gate size k exceeds the number of qubits");
    if (!qubits || !matrix) return fail(CAST_ERR_ARG, "null qubits or matrix");
    uint64_t seen = 0;
    for (int i = 0; i < k; i++) {
        if (qubits[i] < 0 || qubits[i] >= n) return fail(CAST_ERR_ARG, "qubit index out of range");
        uint64_t b = uint64_t(1) << qubits[i];
        if (seen & b) return fail(CAST_ERR_ARG, "duplicate qubit in gate");
        seen |= b;
    }
    for (size_t i = 0; i < (size_t(1) << (2 * k)); i++)
        if (!std::isfinite(matrix[i].real()) || !std::isfinite(matrix[i].imag()))
            return fail(CAST_ERR_ARG, "non-finite matrix entry");

    // order[i] = position in the caller's list of the i-th smallest qubit
    int order[CAST_MAX_K];
    for (int i = 0; i < k; i++) order[i] = i;
    std::sort(order, order + k, [&](int a, int b) { return qubits[a] < qubits[b]; });
    g->k = k;
    for (int i = 0; i < k; i++) g->q[i] = qubits[order[i]];
    const int d = 1 << k;
    std::vector<int> old(d);  // sorted-order index -> caller-order index
    for (int j = 0; j < d; j++) {
        int o = 0;
        for (int i = 0; i < k; i++)
            if ((j >> i) & 1) o |= 1 << order[i];
        old[j] = o;
    }
    g->m.assign(size_t(d) * d, cplx());
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) {
            cplx v = matrix[size_t(old[r]) * d + old[c]];
            double re = std::fabs(v.real()) <= tol ? 0.0 : v.real();
            double im = std::fabs(v.imag()) <= tol ? 0.0 : v.imag();
            g->m[size_t(r) * d + c] = cplx(re, im);
        }

    // unitarity (the tensor-core path relies on it, see apply_tc.cu)
    {
        double worst = 0.0;
        for (int r = 0; r < d && worst <= 1e-9; r++)
            for (int c = 0; c < d; c++) {
                cplx s(0.0, 0.0);
                for (int t = 0; t < d; t++) s += std::conj(g->m[size_t(t) * d + r]) * g->m[size_t(t) * d + c];
                worst = std::max(worst, std::abs(s - (r == c ? cplx(1.0, 0.0) : cplx(0.0, 0.0))));
            }
        g->unitary = worst <= 1e-9;
    }

    // classify: diagonal, monomial (one non-zero per row and column), dense
    bool diag = true;
    for (int r = 0; r < d && diag; r++)
        for (int c = 0; c < d; c++)
            if (r != c && g->m[size_t(r) * d + c] != cplx(0.0, 0.0)) { diag = false; break; }
    if (diag) {
        g->diag.resize(d);
        bool ident = true;
        for (int r = 0; r < d; r++) {
            g->diag[r] = g->m[size_t(r) * d + r];
            if (std::abs(g->diag[r] - cplx(1.0, 0.0)) > tol) ident = false;
        }
        g->cls = ident ? CLS_IDENTITY : CLS_DIAG;
        return CAST_OK;
    }
    std::vector<int> perm(d, -1), colhits(d, 0);
    bool mono = true;
    for (int r = 0; r < d && mono; r++) {
        for (int c = 0; c < d; c++)
            if (g->m[size_t(r) * d + c] != cplx(0.0, 0.0)) {
                if (perm[r] >= 0) { mono = false; break; }
                perm[r] = c;
                colhits[c]++;
            }
        if (perm[r] < 0) mono = false;
    }
    for (int c = 0; c < d && mono; c++)
        if (colhits[c] != 1) mono = false;
    if (mono) {
        g->cls = CLS_MONO;
        g->perm = perm;
        g->phase.resize(d);
        g->unit_phases = true;
        for (int r = 0; r < d; r++) {
            g->phase[r] = g->m[size_t(r) * d + perm[r]];
            if (std::abs(g->phase[r] - cplx(1.0, 0.0)) > tol) g->unit_phases = false;
        }
        return CAST_OK;
    }
    g->cls = CLS_DENSE;
    return CAST_OK;
}

}  // namespace cast
