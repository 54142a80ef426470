// Host planner: canonicalisation, the circuit partition of Algorithm 1
// (Sec. 4.1), greedy gate fusion and the layout of each stage's ops into
// shared-memory tile passes.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <set>

#include "qsim_internal.h"

namespace qsim {

namespace {

bool is_unitary(const std::vector<cd> &u, uint32_t dim) {
    for (uint32_t i = 0; i < dim; ++i)
        for (uint32_t j = 0; j < dim; ++j) {
            cd s = 0;
            for (uint32_t r = 0; r < dim; ++r) s += std::conj(u[r * dim + i]) * u[r * dim + j];
            cd want = (i == j) ? cd(1, 0) : cd(0, 0);
            if (std::abs(s - want) > 1e-8) return false;
        }
    return true;
}

int canonicalize(uint32_t n, const qsim_gate *gates, size_t ngates, std::vector<Gate> *out) {
    out->clear();
    out->reserve(ngates);
    for (size_t i = 0; i < ngates; ++i) {
        const qsim_gate &g = gates[i];
        Gate c;
        if (g.flags & QSIM_GATE_PHASEFLIP) {
            if (n < 64 && (g.basis >> n) != 0)
                return set_error(QSIM_E_INVALID, "gate %zu: phase-flip basis out of range", i);
            c.phaseflip = true;
            c.diag = true;
            c.basis = g.basis;
            c.nq = n;
            out->push_back(std::move(c));
            continue;
        }
        if (g.nq < 1 || g.nq > 6) return set_error(QSIM_E_INVALID, "gate %zu: nq=%u not in 1..6", i, g.nq);
        if (!g.u) return set_error(QSIM_E_INVALID, "gate %zu: matrix is NULL", i);
        c.nq = g.nq;
        for (uint32_t j = 0; j < g.nq; ++j) {
            if (g.q[j] >= n) return set_error(QSIM_E_INVALID, "gate %zu: qubit %u >= n", i, g.q[j]);
            for (uint32_t l = 0; l < j; ++l)
                if (g.q[l] == g.q[j]) return set_error(QSIM_E_INVALID, "gate %zu: repeated qubit", i);
            c.q[j] = g.q[j];
        }
        uint32_t dim = 1u << g.nq;
        c.u.resize(size_t(dim) * dim);
        bool diag = true;
        for (uint32_t r = 0; r < dim; ++r)
            for (uint32_t col = 0; col < dim; ++col) {
                double re = g.u[2 * (r * dim + col)], im = g.u[2 * (r * dim + col) + 1];
                if (!isfinite(re) || !isfinite(im))
                    return set_error(QSIM_E_INVALID, "gate %zu: non-finite matrix entry", i);
                c.u[r * dim + col] = cd(re, im);
                if (r != col && (re != 0.0 || im != 0.0)) diag = false;
            }
        if (!is_unitary(c.u, dim)) return set_error(QSIM_E_INVALID, "gate %zu: matrix is not unitary", i);
        c.diag = diag;
        out->push_back(std::move(c));
    }
    return QSIM_OK;
}

// Global qubits a gate counts toward the stage threshold (Algorithm 1). A
// diagonal gate is block-local whatever its qubits: it counts none when
// diagonal exemption is on, or when its own globals exceed the threshold.
int counted_globals(const Gate &g, uint32_t n, uint32_t m, uint32_t thr, bool diag_exempt,
                    uint64_t *mask) {
    uint64_t s = 0;
    uint32_t cnt = 0;
    if (g.phaseflip) {
        for (uint32_t q = m; q < n; ++q) { s |= 1ull << q; ++cnt; }
    } else {
        for (uint32_t j = 0; j < g.nq; ++j)
            if (g.q[j] >= m) { s |= 1ull << g.q[j]; ++cnt; }
    }
    if (g.diag && (diag_exempt || cnt > thr)) { *mask = 0; return QSIM_OK; }
    if (cnt > thr)
        return set_error(QSIM_E_UNSUPPORTED, "a non-diagonal gate touches %u global qubits (threshold %u)",
                         cnt, thr);
    *mask = s;
    return QSIM_OK;
}

// Commutation-aware order for the stage cut. Two gates must keep their
// circuit order when they share a qubit, unless both are diagonal (diagonal
// gates commute). List scheduling: repeatedly take the earliest gate whose
// ordered predecessors are all placed and whose counted global qubits keep the
// current stage within the threshold; when none fits, the stage is closed and
// the next one starts empty. Every placed gate follows all the gates it does not
// commute with, so the reordered circuit is the same unitary; the in-order cut
// of Algorithm 1 over the new list then yields these stages.
int reorder_for_stages(std::vector<Gate> &gates, uint32_t n, uint32_t m, uint32_t thr, bool diag_exempt) {
    const size_t N = gates.size();
    std::vector<uint64_t> gmask(N);
    std::vector<std::vector<uint32_t>> succ(N);
    std::vector<uint32_t> npred(N, 0);
    {
        std::vector<int64_t> last_nd(n, -1);             // last non-diagonal gate on each qubit
        std::vector<std::vector<uint32_t>> diag_since(n);  // diagonal gates on the qubit since then
        std::vector<uint32_t> preds;
        for (size_t i = 0; i < N; ++i) {
            const Gate &g = gates[i];
            int rc = counted_globals(g, n, m, thr, diag_exempt, &gmask[i]);
            if (rc) return rc;
            std::vector<uint32_t> qs;
            if (g.phaseflip)
                for (uint32_t q = 0; q < n; ++q) qs.push_back(q);
            else
                qs.assign(g.q, g.q + g.nq);
            const bool d = g.diag || g.phaseflip;
            preds.clear();
            for (uint32_t q : qs) {
                if (last_nd[q] >= 0) preds.push_back(uint32_t(last_nd[q]));
                if (!d) preds.insert(preds.end(), diag_since[q].begin(), diag_since[q].end());
            }
            std::sort(preds.begin(), preds.end());
            preds.erase(std::unique(preds.begin(), preds.end()), preds.end());
            for (uint32_t pj : preds) succ[pj].push_back(uint32_t(i));
            npred[i] = uint32_t(preds.size());
            for (uint32_t q : qs) {
                if (d) {
                    diag_since[q].push_back(uint32_t(i));
                } else {
                    last_nd[q] = int64_t(i);
                    diag_since[q].clear();
                }
            }
        }
    }
    std::set<uint32_t> ready;
    for (size_t i = 0; i < N; ++i)
        if (!npred[i]) ready.insert(uint32_t(i));
    std::vector<uint32_t> order;
    order.reserve(N);
    uint64_t mask = 0;
    while (!ready.empty()) {
        uint32_t pick = UINT32_MAX;
        for (uint32_t i : ready)
            if (__builtin_popcountll(mask | gmask[i]) <= int(thr)) { pick = i; break; }
        if (pick == UINT32_MAX) {  // nothing fits: close the stage
            mask = 0;
            continue;
        }
        ready.erase(pick);
        mask |= gmask[pick];
        order.push_back(pick);
        for (uint32_t s2 : succ[pick])
            if (--npred[s2] == 0) ready.insert(s2);
    }
    if (order.size() != N) return set_error(QSIM_E_INVALID, "internal: gate order incomplete");
    std::vector<Gate> out;
    out.reserve(N);
    for (uint32_t i : order) out.push_back(std::move(gates[i]));
    gates.swap(out);
    return QSIM_OK;
}

// Pass-aware order of one stage's gates (QSIM_REORDER_PASSES). Every tile
// pass holds the low L working bits and at most T bits in all; a non-diagonal
// gate needs its qubits among them, a diagonal gate needs none (its phase
// index comes from any bits). List scheduling over the stage's commutation
// order (two gates keep their order when they share a qubit, unless both are
// diagonal), which also shapes the fusion that follows: the next gate is
//   1. a ready non-diagonal gate that joins the dense op being built (the union
//      of their qubits within k, and within the pass's T bits), fewest new op
//      bits first, then fewest new tile bits;
//   2. else a ready diagonal gate inside that op (the fuser folds it in);
//   3. else every ready diagonal gate, placed together (the fuser gathers them
//      into few diagonal ops); the dense op being built ends;
//   4. else a ready non-diagonal gate that starts a new dense op, the one
//      adding the fewest new tile bits;
//   5. else the pass closes and the next one starts from the low L bits.
// Ties go to the gate earliest in the stage. Gates [first, first + count) are
// permuted in place (each gate still follows every gate it does not commute
// with, so the stage is the same unitary); `breaks` receives the
// stage-relative positions where a new pass starts and `masks` the tile bits of
// each pass (breaks.size() + 1 entries). Returns false, leaving the gates as
// they are, if a non-diagonal gate has a qubit outside the working vector
// (which Algorithm 1's cut excludes).
bool pack_stage_passes(std::vector<Gate> &gates, size_t first, size_t count, const std::vector<uint32_t> &inner,
                       uint32_t n, uint32_t m, uint32_t T, uint32_t L, uint32_t k, std::vector<size_t> *breaks,
                       std::vector<uint64_t> *masks) {
    breaks->clear();
    masks->clear();
    auto wbit = [&](uint32_t q) -> int32_t {
        if (q < m) return int32_t(q);
        auto it = std::find(inner.begin(), inner.end(), q);
        return it == inner.end() ? -1 : int32_t(m + (it - inner.begin()));
    };
    if (T > 63 || L > T) return false;
    const uint64_t low = (1ull << L) - 1;
    // need: working bits of a non-diagonal gate; dneed: those of a diagonal gate whose qubits are all
    // working bits (one that a dense op can absorb), else 0
    std::vector<uint64_t> need(count, 0), dneed(count, 0);
    std::vector<char> isdiag(count, 0);
    std::vector<std::vector<uint32_t>> succ(count);
    std::vector<uint32_t> npred(count, 0);
    {
        std::vector<int64_t> last_nd(n, -1);
        std::vector<std::vector<uint32_t>> diag_since(n);
        std::vector<uint32_t> preds, qs;
        for (size_t i = 0; i < count; ++i) {
            const Gate &g = gates[first + i];
            qs.clear();
            if (g.phaseflip)
                for (uint32_t q = 0; q < n; ++q) qs.push_back(q);
            else
                qs.assign(g.q, g.q + g.nq);
            const bool d = g.diag || g.phaseflip;
            isdiag[i] = d;
            if (!d) {
                for (uint32_t q : qs) {
                    const int32_t w = wbit(q);
                    if (w < 0 || w >= 64) return false;
                    need[i] |= 1ull << w;
                }
            } else if (!g.phaseflip) {
                uint64_t dm = 0;
                bool all = true;
                for (uint32_t q : qs) {
                    const int32_t w = wbit(q);
                    if (w < 0 || w >= 64) all = false;
                    else dm |= 1ull << w;
                }
                dneed[i] = all ? dm : 0;
            }
            preds.clear();
            for (uint32_t q : qs) {
                if (last_nd[q] >= 0) preds.push_back(uint32_t(last_nd[q]));
                if (!d) preds.insert(preds.end(), diag_since[q].begin(), diag_since[q].end());
            }
            std::sort(preds.begin(), preds.end());
            preds.erase(std::unique(preds.begin(), preds.end()), preds.end());
            for (uint32_t pj : preds) succ[pj].push_back(uint32_t(i));
            npred[i] = uint32_t(preds.size());
            for (uint32_t q : qs) {
                if (d) {
                    diag_since[q].push_back(uint32_t(i));
                } else {
                    last_nd[q] = int64_t(i);
                    diag_since[q].clear();
                }
            }
        }
    }
    std::set<uint32_t> ready_d, ready_n;
    for (size_t i = 0; i < count; ++i)
        if (!npred[i]) (isdiag[i] ? ready_d : ready_n).insert(uint32_t(i));
    std::vector<uint32_t> order;
    order.reserve(count);
    uint64_t P = low;  // tile bits of the pass being filled
    uint64_t act = 0;  // working bits of the dense op being built
    auto place = [&](uint32_t i) {
        order.push_back(i);
        P |= need[i];
        for (uint32_t s2 : succ[i])
            if (--npred[s2] == 0) (isdiag[s2] ? ready_d : ready_n).insert(s2);
    };
    auto fits = [&](uint32_t i) { return __builtin_popcountll(P | need[i]) <= int(T); };
    while (order.size() < count) {
        uint32_t pick = UINT32_MAX;
        if (act) {
            int best = INT32_MAX;
            for (uint32_t i : ready_n) {  // 1
                if (__builtin_popcountll(act | need[i]) > int(k) || !fits(i)) continue;
                const int cost = 64 * __builtin_popcountll(need[i] & ~act) + __builtin_popcountll(need[i] & ~P);
                if (cost < best) {
                    best = cost;
                    pick = i;
                    if (!cost) break;
                }
            }
            if (pick != UINT32_MAX) {
                ready_n.erase(pick);
                act |= need[pick];
                place(pick);
                continue;
            }
            for (uint32_t i : ready_d)  // 2
                if (dneed[i] && !(dneed[i] & ~act)) {
                    pick = i;
                    break;
                }
            if (pick != UINT32_MAX) {
                ready_d.erase(pick);
                place(pick);
                continue;
            }
        }
        if (!ready_d.empty()) {  // 3
            while (!ready_d.empty()) {
                const uint32_t i = *ready_d.begin();
                ready_d.erase(ready_d.begin());
                place(i);
            }
            act = 0;
            continue;
        }
        int best = INT32_MAX;
        for (uint32_t i : ready_n) {  // 4
            const int add = __builtin_popcountll(need[i] & ~P);
            if (add < best && fits(i)) {
                best = add;
                pick = i;
                if (!add) break;
            }
        }
        if (pick != UINT32_MAX) {
            ready_n.erase(pick);
            act = need[pick];
            place(pick);
            continue;
        }
        // 5; a DAG always has a ready gate, and every gate fits a fresh pass (k + L <= T)
        if (ready_n.empty() || P == low) return false;
        breaks->push_back(order.size());
        masks->push_back(P);
        P = low;
        act = 0;
    }
    masks->push_back(P);
    std::vector<Gate> out;
    out.reserve(count);
    for (uint32_t i : order) out.push_back(std::move(gates[first + i]));
    for (size_t i = 0; i < count; ++i) gates[first + i] = std::move(out[i]);
    return true;
}

// Embed matrix `u` acting on working bits `bits` (matrix bit j <-> bits[j])
// into the space of the ascending working-bit set `S`.
std::vector<cd> embed(const std::vector<cd> &u, const std::vector<uint32_t> &bits,
                      const std::vector<uint32_t> &S) {
    const uint32_t k = bits.size(), K = S.size();
    std::vector<uint32_t> pos(k);
    uint32_t gate_mask = 0;
    for (uint32_t j = 0; j < k; ++j) {
        pos[j] = std::find(S.begin(), S.end(), bits[j]) - S.begin();
        gate_mask |= 1u << pos[j];
    }
    const uint32_t D = 1u << K, d = 1u << k;
    std::vector<cd> out(size_t(D) * D, cd(0, 0));
    for (uint32_t r = 0; r < D; ++r)
        for (uint32_t c = 0; c < D; ++c) {
            if ((r & ~gate_mask) != (c & ~gate_mask)) continue;
            uint32_t rs = 0, cs = 0;
            for (uint32_t j = 0; j < k; ++j) {
                rs |= ((r >> pos[j]) & 1u) << j;
                cs |= ((c >> pos[j]) & 1u) << j;
            }
            out[size_t(r) * D + c] = u[size_t(rs) * d + cs];
        }
    return out;
}

std::vector<cd> matmul(const std::vector<cd> &a, const std::vector<cd> &b, uint32_t D) {
    std::vector<cd> c(size_t(D) * D, cd(0, 0));
    for (uint32_t i = 0; i < D; ++i)
        for (uint32_t l = 0; l < D; ++l) {
            cd x = a[size_t(i) * D + l];
            if (x == cd(0, 0)) continue;
            for (uint32_t j = 0; j < D; ++j) c[size_t(i) * D + j] += x * b[size_t(l) * D + j];
        }
    return c;
}

bool matrix_is_diagonal(const std::vector<cd> &u, uint32_t D) {
    for (uint32_t r = 0; r < D; ++r)
        for (uint32_t c = 0; c < D; ++c)
            if (r != c && u[size_t(r) * D + c] != cd(0, 0)) return false;
    return true;
}

// Greedy fusion in circuit order. Non-diagonal gates grow the active dense op
// while the union of its qubits stays <= k. Diagonal gates are first folded
// back into the pending diagonal op when they commute with every op placed
// after it (their qubits are disjoint from those ops' qubits; diagonal ops and
// phase flips commute with them anyway), up to kMaxDiagQubits qubits; else they
// join the active op; else they open a new pending diagonal op.
struct Fuser {
    const std::vector<uint32_t> *inner;
    uint32_t m, k;
    std::vector<Op> *ops;
    bool active = false;
    std::vector<uint32_t> S;  // ascending working bits
    std::vector<cd> U;
    uint32_t ngates = 0;
    int64_t diag_op = -1;          // index of the pending diagonal op in *ops
    std::set<uint32_t> blockers;   // full qubits of the ops placed after it
    int64_t csep_op = -1;          // index of the pending controlled-separable diagonal op
    std::set<uint32_t> csep_blockers;
    uint32_t last2[2] = {0, 0};    // qubits of the last two-qubit diagonal gate seen
    bool have_last2 = false;
    uint64_t allowed = ~0ull;      // working bits a dense op may take (pass-aware mode: the pass's tile bits)

    int32_t working_bit(uint32_t q) const {
        if (q < m) return int32_t(q);
        auto it = std::find(inner->begin(), inner->end(), q);
        if (it == inner->end()) return -1;
        return int32_t(m + (it - inner->begin()));
    }
    uint32_t qubit_of(uint32_t w) const { return w < m ? w : (*inner)[w - m]; }

    void flush() {
        if (!active) return;
        Op op{};
        const uint32_t D = 1u << S.size();
        op.k = S.size();
        op.ngates = ngates;
        if (matrix_is_diagonal(U, D)) {
            op.type = OP_DIAG;
            for (uint32_t j = 0; j < op.k; ++j) op.fq[j] = qubit_of(S[j]);
            op.u.resize(D);
            for (uint32_t r = 0; r < D; ++r) op.u[r] = U[size_t(r) * D + r];
        } else {
            op.type = OP_DENSE;
            for (uint32_t j = 0; j < op.k; ++j) op.wq[j] = S[j];
            op.u = U;
        }
        for (uint32_t w : S) {
            blockers.insert(qubit_of(w));
            csep_blockers.insert(qubit_of(w));
        }
        ops->push_back(std::move(op));
        active = false;
        S.clear();
        U.clear();
        ngates = 0;
    }

    // ops[diag_op] *= the diagonal gate g (phases multiply; qubit sets unite)
    void fold_diag(const Gate &g) {
        Op &d = (*ops)[size_t(diag_op)];
        std::set<uint32_t> uni(d.fq, d.fq + d.k);
        uni.insert(g.q, g.q + g.nq);
        const std::vector<uint32_t> NQ(uni.begin(), uni.end());
        const uint32_t K = NQ.size(), dg = 1u << g.nq;
        std::vector<cd> nu(size_t(1) << K);
        for (uint32_t x = 0; x < (1u << K); ++x) {
            uint32_t a = 0, b = 0;
            for (uint32_t j = 0; j < K; ++j) {
                const uint32_t bit = (x >> j) & 1u;
                for (uint32_t i = 0; i < d.k; ++i)
                    if (d.fq[i] == NQ[j]) a |= bit << i;
                for (uint32_t i = 0; i < g.nq; ++i)
                    if (g.q[i] == NQ[j]) b |= bit << i;
            }
            nu[x] = d.u[a] * g.u[size_t(b) * dg + b];
        }
        d.k = K;
        for (uint32_t j = 0; j < K; ++j) d.fq[j] = NQ[j];
        d.u = std::move(nu);
        d.ngates += 1;
    }

    // a one- or two-qubit diagonal gate g folded into the pending controlled-separable op
    bool fold_csep(const Gate &g) {
        Op &c = (*ops)[size_t(csep_op)];
        const uint32_t ctl = c.csep_q[0];
        const uint32_t d = 1u << g.nq;
        auto target_index = [&](uint32_t q) -> int64_t {
            for (size_t t = 1; t < c.csep_q.size(); ++t)
                if (c.csep_q[t] == q) return int64_t(t - 1);
            return -1;
        };
        auto add_target = [&](uint32_t q) -> size_t {
            c.csep_q.push_back(q);
            for (int v = 0; v < 4; ++v) c.u.push_back(cd(1, 0));
            return c.csep_q.size() - 2;
        };
        const cd *gd = nullptr;
        std::vector<cd> diag(d);
        for (uint32_t r = 0; r < d; ++r) diag[r] = g.u[size_t(r) * d + r];
        gd = diag.data();
        if (g.nq == 1) {
            if (g.q[0] == ctl) {
                c.u[0] *= gd[0];
                c.u[1] *= gd[1];
            } else {
                int64_t t = target_index(g.q[0]);
                if (t < 0) t = int64_t(add_target(g.q[0]));
                for (int b = 0; b < 2; ++b)
                    for (int x = 0; x < 2; ++x) c.u[2 + 4 * size_t(t) + 2 * b + x] *= gd[x];
            }
        } else {
            // matrix bit 0 <-> g.q[0], bit 1 <-> g.q[1]
            const bool c0 = g.q[0] == ctl;
            const uint32_t tq = c0 ? g.q[1] : g.q[0];
            int64_t t = target_index(tq);
            if (t < 0) t = int64_t(add_target(tq));
            for (int b = 0; b < 2; ++b)
                for (int x = 0; x < 2; ++x) {
                    const uint32_t idx = c0 ? uint32_t(b | (x << 1)) : uint32_t(x | (b << 1));
                    c.u[2 + 4 * size_t(t) + 2 * b + x] *= gd[idx];
                }
        }
        c.k = uint32_t(c.csep_q.size());
        c.ngates += 1;
        return true;
    }

    bool csep_accepts(const Gate &g) const {
        if (csep_op < 0 || g.nq > 2) return false;
        const Op &c = (*ops)[size_t(csep_op)];
        const uint32_t ctl = c.csep_q[0];
        for (uint32_t j = 0; j < g.nq; ++j) {
            if (csep_blockers.count(g.q[j])) return false;
            const int32_t w = working_bit(g.q[j]);
            if (active && w >= 0 && std::find(S.begin(), S.end(), uint32_t(w)) != S.end()) return false;
        }
        if (g.nq == 2) return g.q[0] == ctl || g.q[1] == ctl;
        if (g.q[0] == ctl) return true;
        for (size_t t = 1; t < c.csep_q.size(); ++t)
            if (c.csep_q[t] == g.q[0]) return true;
        return false;
    }

    // the gate joins the active op if the union of qubits stays <= k
    bool try_join(const Gate &g, const std::vector<uint32_t> &wb) {
        std::set<uint32_t> uni(S.begin(), S.end());
        uni.insert(wb.begin(), wb.end());
        if (!active || uni.size() > k) return false;
        for (uint32_t w : uni)
            if (w >= 64 || !((allowed >> w) & 1ull)) return false;
        std::vector<uint32_t> NS(uni.begin(), uni.end());
        std::vector<cd> cur = embed(U, S, NS);
        std::vector<cd> gm = embed(g.u, wb, NS);
        U = matmul(gm, cur, 1u << NS.size());  // later gate on the left
        S = NS;
        ++ngates;
        return true;
    }

    void add(const Gate &g) {
        if (g.phaseflip) {
            // diagonal: the pending diagonal op may still move across it
            flush();
            Op op{};
            op.type = OP_PHASEFLIP;
            op.basis = g.basis;
            op.ngates = 1;
            ops->push_back(std::move(op));
            return;
        }
        std::vector<uint32_t> wb(g.nq);
        bool all_working = true;
        for (uint32_t j = 0; j < g.nq; ++j) {
            int32_t w = working_bit(g.q[j]);
            if (w < 0) all_working = false;
            wb[j] = uint32_t(w);
        }
        if (g.diag) {
            // two-qubit diagonal gates sharing a qubit with the previous one form a star: fold it into a
            // controlled-separable op on the shared qubit
            uint32_t star = 0;
            bool is_star = false;
            if (g.nq == 2) {
                if (have_last2)
                    for (uint32_t a = 0; a < 2; ++a)
                        for (uint32_t b = 0; b < 2; ++b)
                            if (!is_star && g.q[a] == last2[b]) {
                                star = g.q[a];
                                is_star = true;
                            }
                last2[0] = g.q[0];
                last2[1] = g.q[1];
                have_last2 = true;
            }
            bool touches_active = false, commutes = diag_op >= 0;
            for (uint32_t j = 0; j < g.nq; ++j) {
                if (all_working && std::find(S.begin(), S.end(), wb[j]) != S.end()) touches_active = true;
                if (blockers.count(g.q[j])) commutes = false;
                if (active && working_bit(g.q[j]) >= 0 &&
                    std::find(S.begin(), S.end(), uint32_t(working_bit(g.q[j]))) != S.end())
                    commutes = false;
            }
            if (all_working && g.nq <= k && touches_active && try_join(g, wb)) return;
            if (csep_accepts(g)) {
                fold_csep(g);
                return;
            }
            if (commutes) {
                const Op &d = (*ops)[size_t(diag_op)];
                std::set<uint32_t> uni(d.fq, d.fq + d.k);
                uni.insert(g.q, g.q + g.nq);
                if (uni.size() <= kMaxDiagQubits) {
                    fold_diag(g);
                    return;
                }
            }
            if (all_working && g.nq <= k && try_join(g, wb)) return;
            flush();
            if (is_star) {
                Op op{};
                op.type = OP_CSEP;
                op.csep_q.push_back(star);
                op.u = {cd(1, 0), cd(1, 0)};
                op.k = 1;
                op.ngates = 0;
                ops->push_back(std::move(op));
                csep_op = int64_t(ops->size()) - 1;
                csep_blockers.clear();
                fold_csep(g);
                return;
            }
            Op op{};
            op.type = OP_DIAG;
            op.k = g.nq;
            op.ngates = 1;
            const uint32_t d = 1u << g.nq;
            for (uint32_t j = 0; j < g.nq; ++j) op.fq[j] = g.q[j];
            op.u.resize(d);
            for (uint32_t r = 0; r < d; ++r) op.u[r] = g.u[size_t(r) * d + r];
            ops->push_back(std::move(op));
            diag_op = int64_t(ops->size()) - 1;
            blockers.clear();
            return;
        }
        if (try_join(g, wb)) return;
        flush();
        std::set<uint32_t> own(wb.begin(), wb.end());
        S.assign(own.begin(), own.end());
        U = embed(g.u, wb, S);
        ngates = 1;
        active = true;
    }
};

constexpr uint32_t kCoalesceBits = 3;

// A controlled-separable op on at most kMaxDiagQubits qubits becomes an ordinary
// diagonal op (its phase table written out), which the decoder can also apply.
void narrow_csep_ops(std::vector<Op> &ops) {
    for (Op &op : ops) {
        if (op.type != OP_CSEP || op.csep_q.size() > kMaxDiagQubits) continue;
        const uint32_t K = uint32_t(op.csep_q.size());
        std::vector<cd> tab(size_t(1) << K);
        for (uint32_t x = 0; x < (1u << K); ++x) {
            const uint32_t b = x & 1u;  // matrix bit 0 <-> the control
            cd ph = op.u[b];
            for (uint32_t t = 1; t < K; ++t) ph *= op.u[2 + 4 * size_t(t - 1) + 2 * b + ((x >> t) & 1u)];
            tab[x] = ph;
        }
        op.type = OP_DIAG;
        op.k = K;
        for (uint32_t j = 0; j < K; ++j) op.fq[j] = op.csep_q[j];
        op.u = std::move(tab);
        op.csep_q.clear();
    }
}

// shared-memory bytes of an op's data in a pass of 2^T-amplitude tiles: its descriptor; a diagonal op's index
// tables and phases, or, for a polynomial one in a 4096-amplitude tile, its share of the run's summed polynomial
// (832 bytes per run) and term records; a controlled-separable op's tile-bit tables, records and per-tile branch table
size_t pass_op_bytes(const Op &op, uint32_t T) {
    if (op.type == OP_CSEP) return kOpDescBytes + kCsepTableBytes + 48 * size_t(op.k) + 1024;
    if (op.type == OP_DENSE && op.k >= 3 && op.k <= 6)  // tensor-core offset tables: 128 + 2^k words
        return kOpDescBytes + 4 * (128 + (size_t(1) << op.k));
    if (op.type == OP_DIAG && op.quad && T == 12) return kOpDescBytes + 128 + 16 * size_t(op.k);
    return kOpDescBytes + (op.type == OP_DIAG ? 192 + 16 + (size_t(8) << op.k) : 0);
}

void layout_passes(Stage &st, uint32_t tile_bits, bool fold_leading_diag) {
    const uint32_t W = st.W;
    st.pre_ops.clear();
    uint32_t first = 0;
    if (fold_leading_diag) {
        // leading phase ops need no tile: the decoder applies them per element
        while (first < st.ops.size() && (st.ops[first].type == OP_DIAG || st.ops[first].type == OP_PHASEFLIP) &&
               st.pre_ops.size() < kMaxPreOps)
            st.pre_ops.push_back(first++);
    }
    uint32_t T = std::min(tile_bits, W);
    // the low kCoalesceBits working bits are always tile bits: rows of 2^kCoalesceBits amplitudes
    // (64 bytes, two DRAM sectors) are read and written whole
    const uint32_t L = std::min<uint32_t>(kCoalesceBits, T);
    st.passes.clear();
    auto close = [&](std::set<uint32_t> &P, std::vector<uint32_t> &ops) {
        if (ops.empty()) return;
        for (uint32_t b = 0; P.size() < T && b < W; ++b) P.insert(b);
        Pass p{};
        p.T = T;
        uint32_t t = 0;
        for (uint32_t b : P) p.tile_pos[t++] = b;
        p.ops = ops;
        st.passes.push_back(std::move(p));
        ops.clear();
    };
    std::set<uint32_t> P;
    for (uint32_t b = 0; b < L; ++b) P.insert(b);
    std::vector<uint32_t> cur;
    size_t bytes = 0;
    for (uint32_t i = first; i < st.ops.size(); ++i) {
        const Op &op = st.ops[i];
        bool fresh = bytes + pass_op_bytes(op, T) > kPassOpBytes;
        std::set<uint32_t> need(P);
        if (op.type == OP_DENSE) {
            for (uint32_t j = 0; j < op.k; ++j) need.insert(op.wq[j]);
            fresh = fresh || need.size() > T;
        }
        if (fresh && !cur.empty()) {
            close(P, cur);
            P.clear();
            for (uint32_t b = 0; b < L; ++b) P.insert(b);
            bytes = 0;
            if (op.type == OP_DENSE)
                for (uint32_t j = 0; j < op.k; ++j) P.insert(op.wq[j]);
        } else if (op.type == OP_DENSE) {
            P = need;
        }
        bytes += pass_op_bytes(op, T);
        cur.push_back(i);
    }
    close(P, cur);
}

// Modelled time of a stage's tile passes, to choose between two layouts of the same stage (relative units:
// one pass over 2^28 amplitudes, in ms on GB300). A pass costs its load and store plus its ops; the
// coefficients are the k_pass times the ncu launch list gave for 28-qubit QAOA passes of every composition
// (TF32 dense ops of width 3 to 5 on tcgen05; the warp-level MMA form runs these passes at about the same rate):
// with 4 resident CTAs per SM 0.61 per pass and 0.213 per tensor-core dense op; with 3 (a pass whose op data
// pushes a CTA's shared memory past a quarter of the SM's) 0.72 and 0.315 (scaled by the ratio measured before
// the epilogue of the tcgen05 ops changed) and 0.17 per diagonal op applied from a phase table (0.13 with 4
// CTAs, scaled by 3/4); a run of diagonal ops applied as one phase polynomial 0.25 plus 0.055 per op; dense ops
// outside the tensor cores 0.57 (width 1 or 2, measured) or, at width 3 or more, their FP32 arithmetic at the
// CUDA cores' rate (8 * 2^k flops per amplitude at 80 TFLOP/s).
double stage_pass_cost(const Stage &st, const qsim_config *cfg) {
    constexpr double kSmemPerSm = 233472, kStatic = 1250, kReserved = 1024;
    double total = 0;
    for (const Pass &ps : st.passes) {
        const bool tc = cfg->tcgen05 && ps.T == 12 &&
                        (cfg->prec == QSIM_PREC_TF32 || cfg->prec == QSIM_PREC_BF16X3);
        size_t blob = 0, mat = 0, bbytes = 0;
        double d_tc = 0, d_cc = 0, ccw = 0, g = 0, pr = 0, po = 0;
        bool in_poly = false;  // inside a run of polynomial diagonal ops (one sweep for the whole run)
        for (uint32_t oi : ps.ops) {
            const Op &op = st.ops[oi];
            blob += pass_op_bytes(op, ps.T);
            const bool poly = op.type == OP_DIAG && op.quad && ps.T == 12;
            if (poly) {
                if (!in_poly) pr += 1;
                po += 1;
                in_poly = true;
                continue;
            }
            in_poly = false;
            if (op.type == OP_DENSE) {
                // tcgen05 (widths 3 to 5, TF32 also 6), or warp-level MMAs (TF32 widths 3 to 5, split BF16 4
                // and 5), which run these passes at about the same rate
                const uint32_t min_k = cfg->prec == QSIM_PREC_TF32 ? 3u : 4u;
                const bool on_tc = (tc && op.k >= 3 && (op.k <= 5 || cfg->prec == QSIM_PREC_TF32)) ||
                                   (cfg->prec != QSIM_PREC_FP32 && ps.T == 12 && op.k >= min_k && op.k <= 5);
                if (on_tc) {
                    d_tc += 1;
                    bbytes = std::max<size_t>(bbytes, op.k == 6 ? 65536 : cfg->prec == QSIM_PREC_BF16X3 ? 24576 : 16384);
                } else if (op.k <= 2) {
                    d_cc += 1;
                    mat = std::max<size_t>(mat, size_t(8) << (2 * op.k));
                } else {
                    ccw += double(uint64_t(8) << op.k) * double(1ull << 28) / 80e12 * 1e3;
                    mat = std::max<size_t>(mat, size_t(8) << (2 * op.k));
                }
            } else if (op.type == OP_DIAG || op.type == OP_CSEP) {
                g += 1;
            }
        }
        const double smem = double(size_t(8) << ps.T) + (bbytes ? double(bbytes) + 1024 : 0) + double(blob + mat) +
                            kStatic + kReserved;
        const int ctas = std::max(1, std::min(4, int(kSmemPerSm / smem)));
        const double polys = 0.25 * pr + 0.055 * po;
        if (ctas >= 4)
            total += 0.61 + 0.213 * d_tc + 0.13 * g + 0.57 * d_cc + ccw + polys;
        else
            total += (0.72 + 0.315 * d_tc + 0.17 * g + 0.57 * d_cc + ccw) * (3.0 / ctas) + polys;
    }
    return total;
}

}  // namespace

bool diag_quadratic(const Op &op, DiagPoly *out) {
    if (op.type != OP_DIAG || op.k > 8 || op.u.size() != (size_t(1) << op.k)) return false;
    const uint32_t K = op.k, D = 1u << K;
    const double two_pi = 6.283185307179586476925286766559;
    auto red = [](double t) { return t - std::floor(t + 0.5); };  // to [-1/2, 1/2)
    std::vector<double> ph(D);
    for (uint32_t x = 0; x < D; ++x) {
        if (std::fabs(std::abs(op.u[x]) - 1.0) > 1e-9) return false;
        ph[x] = std::arg(op.u[x]) / two_pi;
    }
    DiagPoly q;
    q.c = ph[0];
    for (uint32_t j = 0; j < K; ++j) q.a[j] = red(ph[1u << j] - q.c);
    for (uint32_t j = 0; j < K; ++j)
        for (uint32_t l = j + 1; l < K; ++l)
            q.g[j][l] = red(ph[(1u << j) | (1u << l)] - ph[1u << j] - ph[1u << l] + q.c);
    for (uint32_t x = 0; x < D; ++x) {
        double t = q.c;
        for (uint32_t j = 0; j < K; ++j) {
            if (!((x >> j) & 1u)) continue;
            t += q.a[j];
            for (uint32_t l = j + 1; l < K; ++l)
                if ((x >> l) & 1u) t += q.g[j][l];
        }
        if (std::fabs(red(ph[x] - t)) > 1e-9) return false;
    }
    q.c = red(q.c);
    *out = q;
    return true;
}

bool qsz_step_exponent(double eb, int *e) {
    if (!(eb > 0.0) || !isfinite(eb)) return false;
    int x;
    (void)frexp(2.0 * eb, &x);
    int v = x - 1;
    if (v < kQszEMin || v > kQszEMax) return false;
    *e = v;
    return true;
}

bool qszr_shift(double rel, int *k) {
    if (!(rel > 0.0) || !(rel < 1.0)) return false;
    const double r = rel / (1.0 + rel);
    int x;
    (void)frexp(std::ldexp(r, 24), &x);  // 2^24 r = f 2^x, f in [0.5, 1)
    int v = x - 1;
    while (v >= kQszrKMin && std::ldexp(1.0, v - 24) > r) --v;
    if (v < kQszrKMin || v > kQszrKMax) return false;
    *k = v;
    return true;
}

int build_plan(uint32_t n, const qsim_gate *gates, size_t ngates, const qsim_config *cfg,
               qsim_plan **out) {
    auto t0 = std::chrono::steady_clock::now();
    if (!out || !cfg) return set_error(QSIM_E_INVALID, "null argument");
    *out = nullptr;
    if (n < 5 || n > 40) return set_error(QSIM_E_INVALID, "n=%u not in 5..40", n);
    if (cfg->m < uint32_t(kQszMinM) || cfg->m > uint32_t(kQszMaxM) || cfg->m > n)
        return set_error(QSIM_E_INVALID, "m=%u not in 5..min(26, n)", cfg->m);
    if (cfg->k < 1 || cfg->k > 6) return set_error(QSIM_E_INVALID, "k=%u not in 1..6", cfg->k);
    if (cfg->prec > QSIM_PREC_BF16X3) return set_error(QSIM_E_INVALID, "bad precision %u", cfg->prec);
    if (cfg->tcgen05 > 1) return set_error(QSIM_E_INVALID, "tcgen05 is 0 or 1");
    if (cfg->reorder > QSIM_REORDER_PASSES_ALL) return set_error(QSIM_E_INVALID, "reorder is 0 to 3");
    if (cfg->mode > QSIM_MODE_PERSISTENT) return set_error(QSIM_E_INVALID, "bad mode %u", cfg->mode);
    if (cfg->mode == QSIM_MODE_PERSISTENT && cfg->k > 5 && !(cfg->tcgen05 && cfg->prec == QSIM_PREC_TF32))
        return set_error(QSIM_E_INVALID, "persistent mode fuses k = 6 only as TF32 on tcgen05");
    if (cfg->codec > QSIM_CODEC_QSZR) return set_error(QSIM_E_INVALID, "bad codec %u", cfg->codec);
    if (cfg->sizing > QSIM_SIZING_PREDICT) return set_error(QSIM_E_INVALID, "bad sizing %u", cfg->sizing);
    if (cfg->mode == QSIM_MODE_STREAMS && (cfg->streams < 1 || cfg->streams > 16))
        return set_error(QSIM_E_INVALID, "streams=%u not in 1..16", cfg->streams);
    if (n < 64 && (cfg->init_basis >> n) != 0) return set_error(QSIM_E_INVALID, "init_basis out of range");
    if (cfg->codec == QSIM_CODEC_QSZ1) {
        int e;
        double eb = cfg->eps * pow(2.0, -double(n) / 2.0);
        if (!qsz_step_exponent(eb, &e)) return set_error(QSIM_E_INVALID, "eps gives an error bound out of range");
    }
    if (cfg->codec == QSIM_CODEC_QSZR) {
        int k;
        if (!qszr_shift(cfg->eps, &k)) return set_error(QSIM_E_INVALID, "relative bound eps out of range");
    }
    if (ngates && !gates) return set_error(QSIM_E_INVALID, "gates is NULL");

    qsim_plan *p = new (std::nothrow) qsim_plan();
    if (!p) return set_error(QSIM_E_NOMEM, "plan allocation");
    p->n = n;
    p->cfg = *cfg;
    int rc = canonicalize(n, gates, ngates, &p->gates);
    if (rc) { delete p; return rc; }

    const uint32_t m = cfg->m;
    const uint32_t thr = std::max<uint32_t>(cfg->inner, 2);
    for (size_t i = 0; i < p->gates.size(); ++i) {
        const Gate &g = p->gates[i];
        if (!g.phaseflip && !g.diag && g.nq > cfg->k) {
            delete p;
            return set_error(QSIM_E_INVALID, "gate %zu is %u-qubit but k=%u", i, g.nq, cfg->k);
        }
    }

    // ---- optional commutation-aware order (stages are then cut from the reordered list) ----
    if (cfg->reorder) {
        rc = reorder_for_stages(p->gates, n, m, thr, cfg->diag_exempt != 0);
        if (rc) { delete p; return rc; }
    }

    // ---- Algorithm 1: greedy in-order partition ----
    uint64_t cur_mask = 0;
    size_t cur_first = 0, cur_count = 0;
    auto emit = [&](uint64_t mask) {
        Stage st;
        st.first_gate = cur_first;
        st.ngates = cur_count;
        for (uint32_t q = m; q < n; ++q)
            if ((mask >> q) & 1) st.inner.push_back(q);
        st.W = m + st.inner.size();
        p->stages.push_back(std::move(st));
    };
    for (size_t i = 0; i < p->gates.size(); ++i) {
        uint64_t gm;
        rc = counted_globals(p->gates[i], n, m, thr, cfg->diag_exempt != 0, &gm);
        if (rc) { delete p; return rc; }
        if (cur_count && __builtin_popcountll(cur_mask | gm) > int(thr)) {
            emit(cur_mask);
            cur_mask = 0;
            cur_first = i;
            cur_count = 0;
        }
        cur_mask |= gm;
        ++cur_count;
    }
    if (cur_count) emit(cur_mask);

    // ---- fusion and tile passes per stage ----
    const uint32_t tile_bits = cfg->tile_bits ? cfg->tile_bits : 12;
    if (tile_bits < 6 || tile_bits > 13) { delete p; return set_error(QSIM_E_INVALID, "tile_bits must be 6..13"); }
    // the stage's gates fused into ops (greedily, in the given order) and laid out in tile passes; with breaks,
    // the fuser closes its dense op at each pass boundary and builds dense ops only from that pass's tile bits
    auto fuse_layout = [&](Stage &st, uint32_t T, const std::vector<size_t> *breaks,
                           const std::vector<uint64_t> *masks) {
        st.ops.clear();
        Fuser fz;
        fz.inner = &st.inner;
        fz.m = m;
        fz.k = cfg->k;
        fz.ops = &st.ops;
        size_t nb = 0;
        if (breaks) fz.allowed = (*masks)[0];
        for (size_t i = 0; i < st.ngates; ++i) {
            if (breaks && nb < breaks->size() && i == (*breaks)[nb]) {
                fz.flush();
                fz.allowed = (*masks)[++nb];
            }
            fz.add(p->gates[st.first_gate + i]);
        }
        fz.flush();
        narrow_csep_ops(st.ops);
        for (Op &op : st.ops) {
            DiagPoly q;
            op.quad = op.type == OP_DIAG && diag_quadratic(op, &q);
        }
        // leading phase ops go to the decoder of either compressed format (the raw copy-in applies none)
        layout_passes(st, T, cfg->codec != QSIM_CODEC_NONE);
    };
    for (Stage &st : p->stages) {
        const uint32_t T = std::max<uint32_t>(tile_bits, std::min<uint32_t>(st.W, 5 + cfg->k));
        fuse_layout(st, T, nullptr, nullptr);
        if (cfg->reorder < QSIM_REORDER_PASSES) continue;
        // pass-aware order: kept when its modelled pass time is at least 5 % below that of the partition order's
        // layout (the model is within about 5 % of most measured passes; closer calls keep the partition order),
        // or in every stage with QSIM_REORDER_PASSES_ALL
        const std::vector<Gate> keep(p->gates.begin() + st.first_gate, p->gates.begin() + st.first_gate + st.ngates);
        std::vector<size_t> breaks;
        std::vector<uint64_t> masks;
        if (!pack_stage_passes(p->gates, st.first_gate, st.ngates, st.inner, n, m, std::min(T, st.W),
                               std::min(kCoalesceBits, std::min(T, st.W)), cfg->k, &breaks, &masks))
            continue;
        Stage packed = st;
        fuse_layout(packed, T, &breaks, &masks);
        if (cfg->reorder == QSIM_REORDER_PASSES_ALL || stage_pass_cost(packed, cfg) < 0.95 * stage_pass_cost(st, cfg)) {
            st = std::move(packed);
            st.pass_order = true;
        } else {
            std::copy(keep.begin(), keep.end(), p->gates.begin() + st.first_gate);
        }
    }

    qsim_plan_stats &s = p->stats;
    s.nstages = p->stages.size();
    s.ngates = p->gates.size();
    for (const Stage &st : p->stages) {
        for (const Op &op : st.ops) {
            if (op.type == OP_DENSE) ++s.dense_ops;
            else if (op.type == OP_DIAG || op.type == OP_CSEP) ++s.diag_ops;
            else ++s.phaseflip_ops;
        }
        s.passes += st.passes.size();
        s.max_working_log2 = std::max<uint64_t>(s.max_working_log2, st.W);
    }
    s.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return QSIM_OK;
}

// Group sharding over 2^r ranks (Sec. 4.2: the SV groups of a stage are independent; Sec. 5.8 runs them on
// several GPUs). Stage s deals its groups by r rank qubits, global qubits outside the stage's inner set, so each
// group, and each of its blocks, sits on the rank numbered by the block's bits at those qubits (rank bit j = the
// bit of rank qubit j). A rank qubit keeps its slot until a stage takes it as an inner qubit; it is then replaced
// by the free global qubit whose next use as an inner qubit is farthest away (never used: farthest of all), so
// blocks move between ranks only at the stage boundaries that need it, and only over the replaced bits.
int plan_shards(const qsim_plan *p, uint32_t r, uint32_t *rank_qubits) {
    if (!p || (r && !rank_qubits)) return set_error(QSIM_E_INVALID, "null argument");
    const uint32_t n = p->n, m = p->cfg.m, ns = uint32_t(p->stages.size());
    if (r == 0 || ns == 0) return QSIM_OK;
    if (r > 16) return set_error(QSIM_E_INVALID, "at most 2^16 ranks");
    auto inner_of = [&](uint32_t s, uint32_t q) {
        const std::vector<uint32_t> &in = p->stages[s].inner;
        return std::find(in.begin(), in.end(), q) != in.end();
    };
    // next stage >= s that takes q as an inner qubit (ns: none)
    auto next_use = [&](uint32_t s, uint32_t q) {
        for (uint32_t t = s; t < ns; ++t)
            if (inner_of(t, q)) return t;
        return ns;
    };
    std::vector<uint32_t> cur;
    for (uint32_t s = 0; s < ns; ++s) {
        if (n - m < r + uint32_t(p->stages[s].inner.size()))
            return set_error(QSIM_E_INVALID, "stage %u: %u global qubits, %zu inner, too few left for %u rank qubits",
                             s, n - m, p->stages[s].inner.size(), r);
        std::vector<uint32_t> next(cur);
        if (next.empty()) next.assign(r, ~0u);
        for (uint32_t j = 0; j < r; ++j) {
            if (next[j] != ~0u && !inner_of(s, next[j])) continue;
            // the free global qubit (not inner now, not held by another slot) used as inner farthest ahead;
            // ties go to the lowest qubit
            uint32_t best = ~0u, best_use = 0;
            for (uint32_t q = m; q < n; ++q) {
                if (inner_of(s, q) || std::find(next.begin(), next.end(), q) != next.end()) continue;
                const uint32_t u = next_use(s, q);
                if (best == ~0u || u > best_use) {
                    best = q;
                    best_use = u;
                }
            }
            next[j] = best;
        }
        for (uint32_t j = 0; j < r; ++j) rank_qubits[size_t(s) * r + j] = next[j];
        cur = next;
    }
    return QSIM_OK;
}

}  // namespace qsim
