// Autotuner: chooses (m, k, inner size, streams) by timing runs of a circuit
// prefix through the library's own entry points, with an in-memory cache.
// The paper studies inner size and SV block size by hand on one workload
// (Sec. 5.8: larger values mean fewer stages and fewer launches); this makes
// the choice per circuit and per machine.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qsim_internal.h"

namespace qsim {
namespace {

std::mutex g_tune_mu;
std::map<std::string, qsim_config> g_tune_cache;

// key: n, every gate's arity, flags and qubits (not its angles), the space and the settings that matter
std::string tune_key(uint32_t n, const qsim_gate *g, size_t ng, const qsim_config *b, const qsim_tune_space *sp) {
    std::string k;
    auto put = [&](uint64_t v) { k.append(reinterpret_cast<const char *>(&v), sizeof(v)); };
    put(n);
    put(ng);
    for (size_t i = 0; i < ng; ++i) {
        put(uint64_t(g[i].nq) | (uint64_t(g[i].flags) << 8));
        const uint32_t nq = (g[i].flags & QSIM_GATE_PHASEFLIP) ? 0 : g[i].nq;
        for (uint32_t j = 0; j < nq && j < 6; ++j) put(g[i].q[j]);
    }
    put(b->prec);
    put(b->codec);
    put(b->sizing);
    put(b->mode);
    put(uint64_t(b->eps * 1e12));
    k.append(reinterpret_cast<const char *>(sp), sizeof(*sp));
    return k;
}

// time one candidate on the prefix; returns +inf when the candidate is not valid for this circuit
double time_candidate(uint32_t n, const qsim_gate *g, size_t ng, const qsim_config &cfg, uint32_t reps) {
    qsim_plan *plan = nullptr;
    if (qsim_plan_stages(n, g, ng, &cfg, &plan) != QSIM_OK) return 1e300;
    double best = 1e300;
    for (uint32_t r = 0; r < std::max<uint32_t>(1, reps) + 1; ++r) {  // first run warms caches
        qsim_state *st = nullptr;
        qsim_stats stats;
        if (qsim_run(plan, nullptr, &st, &stats) != QSIM_OK) {
            best = 1e300;
            break;
        }
        if (r > 0) best = std::min(best, stats.seconds);
        qsim_state_free(st);
    }
    qsim_plan_free(plan);
    return best;
}

}  // namespace
}  // namespace qsim

using namespace qsim;

extern "C" int qsim_autotune(uint32_t n, const qsim_gate *gates, size_t ngates, const qsim_config *base,
                             const qsim_tune_space *space, qsim_config *best, double *best_seconds,
                             uint32_t *candidates) {
    if (!base || !space || !best || (ngates && !gates)) return set_error(QSIM_E_INVALID, "null argument");
    if (space->m_min > space->m_max || space->k_min > space->k_max || space->inner_min > space->inner_max ||
        !(space->streams_mask & 0x1FFFEu))
        return set_error(QSIM_E_INVALID, "empty search space");
    const size_t ng = space->prefix_gates ? std::min<size_t>(ngates, space->prefix_gates) : ngates;
    const std::string key = tune_key(n, gates, ng, base, space);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = it->second;
            if (candidates) *candidates = 0;
            if (best_seconds) *best_seconds = 0;
            return QSIM_OK;
        }
    }
    qsim_config cur = *base;
    auto clampu = [](uint32_t v, uint32_t lo, uint32_t hi) { return std::min(std::max(v, lo), hi); };
    cur.m = clampu(cur.m ? cur.m : 22, space->m_min, std::min<uint32_t>(space->m_max, n));
    cur.k = clampu(cur.k ? cur.k : 5, space->k_min, space->k_max);
    cur.inner = clampu(cur.inner, space->inner_min, space->inner_max);
    const uint32_t wmax = space->max_working_log2;
    auto fits = [&](const qsim_config &c) { return !wmax || c.m + c.inner <= wmax; };
    while (!fits(cur) && cur.inner > space->inner_min) --cur.inner;
    while (!fits(cur) && cur.m > space->m_min) --cur.m;
    if (!fits(cur)) return set_error(QSIM_E_INVALID, "no candidate within the working-vector limit");
    uint32_t s0 = cur.streams;
    if (!(space->streams_mask & (1u << s0))) {
        s0 = 1;
        while (!(space->streams_mask & (1u << s0))) ++s0;
    }
    cur.streams = s0;
    uint32_t timed = 0;
    double cur_t = time_candidate(n, gates, ng, cur, space->reps);
    ++timed;
    auto sweep = [&](uint32_t qsim_config::*field, uint32_t lo, uint32_t hi, uint32_t mask) {
        for (uint32_t v = lo; v <= hi; ++v) {
            if (mask && !(mask & (1u << v))) continue;
            if (v == cur.*field) continue;
            qsim_config c = cur;
            c.*field = v;
            if (!fits(c)) continue;
            const double t = time_candidate(n, gates, ng, c, space->reps);
            ++timed;
            if (t < cur_t) {
                cur_t = t;
                cur = c;
            }
        }
    };
    sweep(&qsim_config::m, space->m_min, std::min<uint32_t>(space->m_max, n), 0);
    sweep(&qsim_config::k, space->k_min, space->k_max, 0);
    sweep(&qsim_config::inner, space->inner_min, space->inner_max, 0);
    sweep(&qsim_config::streams, 1, 16, space->streams_mask);
    if (cur_t >= 1e300) return set_error(QSIM_E_UNSUPPORTED, "no candidate configuration ran");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = cur;
    }
    *best = cur;
    if (best_seconds) *best_seconds = cur_t;
    if (candidates) *candidates = timed;
    return QSIM_OK;
}

extern "C" void qsim_autotune_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
}
