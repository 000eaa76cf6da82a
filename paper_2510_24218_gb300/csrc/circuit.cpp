// Circuit construction (App. A gate lists, App. D QAOA) and error reporting.
#include <cmath>
#include <cstring>
#include <new>

#include "pw_internal.h"

namespace pw {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

bool is_diagonal(const cd* A, int dim) {
    for (int r = 0; r < dim; ++r)
        for (int c = 0; c < dim; ++c)
            if (r != c && A[r * dim + c] != cd(0.0, 0.0)) return false;
    return true;
}

bool is_monomial(const cd* A, int dim) {
    for (int r = 0; r < dim; ++r) {
        int nr = 0, nc = 0;
        for (int c = 0; c < dim; ++c) {
            if (A[r * dim + c] != cd(0.0, 0.0)) ++nr;
            if (A[c * dim + r] != cd(0.0, 0.0)) ++nc;
        }
        if (nr != 1 || nc != 1) return false;
    }
    return true;
}

static bool finite_all(const double* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

static int check_qubits(const pw_circuit* c, int m, const int* qubits) {
    if (!qubits) return set_error(PW_ERR_ARG, "qubits is null");
    for (int i = 0; i < m; ++i) {
        if (qubits[i] < 0 || qubits[i] >= c->n) return set_error(PW_ERR_ARG, "qubit index out of range");
        for (int j = 0; j < i; ++j)
            if (qubits[i] == qubits[j]) return set_error(PW_ERR_ARG, "repeated qubit in one operation");
    }
    return PW_OK;
}

// 2x2 submonomial test: at most one nonzero per row and column.
static bool submonomial2(const cd* M) {
    bool a = M[0] != cd(0, 0), b = M[1] != cd(0, 0), c = M[2] != cd(0, 0), d = M[3] != cd(0, 0);
    return !(a && b) && !(c && d) && !(a && c) && !(b && d);
}

// Tensor-product factorisation of an LSM operator (App. A), local index b0 + 2 b1.
bool lsm_factor(const cd* E, int m, cd* M0, cd* M1) {
    if (m == 1) {
        for (int i = 0; i < 4; ++i) M0[i] = E[i];
        return submonomial2(M0);
    }
    int r = 0, c = 0;
    double best = -1;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            if (std::abs(E[i * 4 + j]) > best) { best = std::abs(E[i * 4 + j]); r = i; c = j; }
    if (best <= 0) return false;
    int r0 = r & 1, r1 = r >> 1, c0 = c & 1, c1 = c >> 1;
    cd piv = E[r * 4 + c];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            M0[a * 2 + b] = E[(a + 2 * r1) * 4 + (b + 2 * c1)];
            M1[a * 2 + b] = E[(r0 + 2 * a) * 4 + (c0 + 2 * b)] / piv;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cd v = M1[(i >> 1) * 2 + (j >> 1)] * M0[(i & 1) * 2 + (j & 1)];
            if (std::abs(v - E[i * 4 + j]) > 1e-13 * (1.0 + std::abs(E[i * 4 + j]))) return false;
        }
    return submonomial2(M0) && submonomial2(M1);
}

}  // namespace pw

using namespace pw;

extern "C" {

const char* pw_last_error(void) { return g_last_error.c_str(); }

int pw_circuit_create(int n_qubits, pw_circuit** out) {
    if (!out) return set_error(PW_ERR_ARG, "out is null");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 4096) return set_error(PW_ERR_ARG, "n_qubits must be in 1..4096");
    pw_circuit* c = new (std::nothrow) pw_circuit();
    if (!c) return set_error(PW_ERR_OOM, "allocation failed");
    c->n = n_qubits;
    *out = c;
    return PW_OK;
}

int pw_circuit_add_gate(pw_circuit* c, int m, const int* qubits, const double* A) {
    if (!c || !A) return set_error(PW_ERR_ARG, "null argument");
    if (m < 1 || m > 2) return set_error(PW_ERR_UNSUPPORTED, "gates act on 1 or 2 qubits");
    int rc = check_qubits(c, m, qubits);
    if (rc) return rc;
    int dim = 1 << m;
    if (!finite_all(A, (size_t)2 * dim * dim)) return set_error(PW_ERR_NUMERIC, "non-finite gate entry");
    Op op;
    op.kind = OP_GATE;
    op.qubits.assign(qubits, qubits + m);
    op.k = 1;
    op.mats.resize((size_t)dim * dim);
    for (int i = 0; i < dim * dim; ++i) op.mats[i] = cd(A[2 * i], A[2 * i + 1]);
    c->ops.push_back(std::move(op));
    return PW_OK;
}

int pw_circuit_add_kraus(pw_circuit* c, int m, const int* qubits, int k, const double* E) {
    if (!c || !E) return set_error(PW_ERR_ARG, "null argument");
    if (m < 1 || m > 2) return set_error(PW_ERR_UNSUPPORTED, "channels act on 1 or 2 qubits");
    if (k < 1 || k > 64) return set_error(PW_ERR_ARG, "k must be in 1..64");
    int rc = check_qubits(c, m, qubits);
    if (rc) return rc;
    int dim = 1 << m;
    if (!finite_all(E, (size_t)2 * k * dim * dim)) return set_error(PW_ERR_NUMERIC, "non-finite Kraus entry");
    Op op;
    op.kind = OP_KRAUS;
    op.qubits.assign(qubits, qubits + m);
    op.k = k;
    op.mats.resize((size_t)k * dim * dim);
    for (size_t i = 0; i < op.mats.size(); ++i) op.mats[i] = cd(E[2 * i], E[2 * i + 1]);
    for (int i = 0; i < k; ++i) {
        cd M0[4], M1[4];
        if (!lsm_factor(op.mat(i), m, M0, M1))
            return set_error(PW_ERR_NOT_LSM, "Kraus operator is not local-submonomial");
    }
    c->ops.push_back(std::move(op));
    return PW_OK;
}

int pw_circuit_num_ops(const pw_circuit* c, int* n_ops) {
    if (!c || !n_ops) return set_error(PW_ERR_ARG, "null argument");
    *n_ops = (int)c->ops.size();
    return PW_OK;
}

void pw_circuit_destroy(pw_circuit* c) { delete c; }

int pw_circuit_qaoa(int n, int n_edges, const int* edges, const double* w, const double* h, int p,
                    const double* gammas, const double* betas, double depol2, double ad_gamma,
                    pw_circuit** out) {
    if (!out) return set_error(PW_ERR_ARG, "out is null");
    *out = nullptr;
    if (n_edges < 0 || p < 0 || (n_edges > 0 && (!edges || !w)) || (p > 0 && (!gammas || !betas)))
        return set_error(PW_ERR_ARG, "bad QAOA arguments");
    if (!(depol2 >= 0.0 && depol2 <= 1.0) || !(ad_gamma >= 0.0 && ad_gamma <= 1.0))
        return set_error(PW_ERR_ARG, "noise strengths must be in [0,1]");
    pw_circuit* c = nullptr;
    int rc = pw_circuit_create(n, &c);
    if (rc) return rc;
    const double s2 = 1.0 / std::sqrt(2.0);
    auto fail = [&](int code) { pw_circuit_destroy(c); return code; };
    // |+>^n
    for (int q = 0; q < n; ++q) {
        double H[8] = {s2, 0, s2, 0, s2, 0, -s2, 0};
        if ((rc = pw_circuit_add_gate(c, 1, &q, H))) return fail(rc);
    }
    // Kraus lists
    std::vector<double> dep, ad;
    if (depol2 > 0) {
        // Paulis I, X, Y, Z as 2x2 complex
        const cd P[4][4] = {{1, 0, 0, 1}, {0, 1, 1, 0}, {0, cd(0, -1), cd(0, 1), 0}, {1, 0, 0, -1}};
        dep.resize(16 * 16 * 2);
        for (int kk = 0; kk < 16; ++kk) {
            int a = kk % 4, b = kk / 4;
            double sc = kk == 0 ? std::sqrt(1.0 - depol2) : std::sqrt(depol2 / 15.0);
            for (int r = 0; r < 4; ++r)
                for (int cc = 0; cc < 4; ++cc) {
                    // kron(P_b, P_a): row = r0 + 2 r1 with r0 on u (Pauli a), r1 on v (Pauli b)
                    cd v = sc * P[b][(r >> 1) * 2 + (cc >> 1)] * P[a][(r & 1) * 2 + (cc & 1)];
                    dep[(kk * 16 + r * 4 + cc) * 2] = v.real();
                    dep[(kk * 16 + r * 4 + cc) * 2 + 1] = v.imag();
                }
        }
    }
    if (ad_gamma > 0) {
        ad.assign(2 * 4 * 2, 0.0);
        ad[0] = 1.0;                                   // E0[0][0]
        ad[6] = std::sqrt(1.0 - ad_gamma);             // E0[1][1]
        ad[8 + 2] = std::sqrt(ad_gamma);               // E1[0][1]
    }
    for (int l = 0; l < p; ++l) {
        double g = gammas[l], b = betas[l];
        if (!std::isfinite(g) || !std::isfinite(b)) return fail(set_error(PW_ERR_NUMERIC, "non-finite angle"));
        for (int e = 0; e < n_edges; ++e) {
            int q[2] = {edges[2 * e], edges[2 * e + 1]};
            double th = 2.0 * g * w[e];
            double D[32] = {0};
            for (int bb = 0; bb < 4; ++bb) {
                int par = (bb & 1) ^ (bb >> 1);
                double ph = -0.5 * th * (par ? -1.0 : 1.0);
                D[(bb * 4 + bb) * 2] = std::cos(ph);
                D[(bb * 4 + bb) * 2 + 1] = std::sin(ph);
            }
            if ((rc = pw_circuit_add_gate(c, 2, q, D))) return fail(rc);
            if (depol2 > 0 && (rc = pw_circuit_add_kraus(c, 2, q, 16, dep.data()))) return fail(rc);
        }
        if (h) {
            for (int j = 0; j < n; ++j) {
                double th = 2.0 * g * h[j];
                double D[8] = {std::cos(-0.5 * th), std::sin(-0.5 * th), 0, 0, 0, 0, std::cos(0.5 * th),
                               std::sin(0.5 * th)};
                if ((rc = pw_circuit_add_gate(c, 1, &j, D))) return fail(rc);
            }
        }
        for (int j = 0; j < n; ++j) {
            double cb = std::cos(b), sb = std::sin(b);   // RX(2 beta) = exp(-i beta X)
            double R[8] = {cb, 0, 0, -sb, 0, -sb, cb, 0};
            if ((rc = pw_circuit_add_gate(c, 1, &j, R))) return fail(rc);
        }
        if (ad_gamma > 0)
            for (int j = 0; j < n; ++j)
                if ((rc = pw_circuit_add_kraus(c, 1, &j, 2, ad.data()))) return fail(rc);
    }
    *out = c;
    return PW_OK;
}

}  // extern "C"
