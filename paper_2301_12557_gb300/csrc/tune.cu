// Measured autotuner: cell side, i-points per thread and histogram privatisation.
//
// The cost model of Appendix B.1 (pc_suggest_cell_size) gives a starting cell
// side; the tuner times the FP32 pair kernel (plus rescue) on an evenly spaced
// sample of the point blocks -- the block-shard mechanism of the multi-GPU
// path with one shard -- first for 2 and 4 i-points per thread at that side,
// then at cell sides in quarter-octave steps from 0.7 to 2 times it, then
// with one count copy per warp, then with the near-edge pairs evaluated
// inside the pair kernel instead of queued, and returns the fastest
// combination.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pc_host.hpp"

using namespace pc;

namespace {

// Largest separation any bin can hold (Sect. 2.5: sqrt(sigma^2 + pi^2) for
// (sigma, pi) bins).
double bins_reach(const pc_bins *b) {
    const double a = b->edges_a[b->n_a];
    if (b->mode == PC_BIN_SIGPI) {
        const double p = b->edges_b[b->n_b];
        return sqrt(a * a + p * p);
    }
    return a;
}

// Cells per axis the grid build would use for a cell side c (before its
// periodic no-alias adjustment, which is the same for equal inputs).
void grid_dims(const pc_box *box, const double lo[3], const double hi[3], double c, long long ng[3]) {
    for (int a = 0; a < 3; ++a) {
        const double ext = hi[a] - lo[a];
        ng[a] = box->periodic ? std::max(1LL, (long long)floor(ext / c))
                              : std::max(1LL, (long long)ceil(ext / c));
    }
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

}  // namespace

extern "C" pc_status pc_tune(const double *xyz, const void *w, int w_is_f32, long long n,
                             const pc_box *box, const pc_bins *b, const pc_opts *base,
                             void *stream, pc_opts *out, pc_tune_trial *trials, int max_trials,
                             int *n_trials) {
    if (n_trials) *n_trials = 0;
    if (!box || !b || !out || n < 0 || (n > 0 && !xyz) || max_trials < 0 ||
        (max_trials > 0 && !trials))
        return fail(PC_EINVAL, "pc_tune: bad arguments");
    if (b->n_a < 1 || !b->edges_a || (b->mode != PC_BIN_S && (b->n_b < 1 || !b->edges_b)))
        return fail(PC_EINVAL, "pc_tune: bad bins");
    pc_opts o;
    memset(&o, 0, sizeof(o));
    if (base) o = *base;
    const double reach = bins_reach(b);
    if (!(reach > 0.0) || !std::isfinite(reach)) return fail(PC_EINVAL, "pc_tune: bad bins");
    cudaStream_t st = (cudaStream_t)stream;

    double lo[3], hi[3];
    const bool given = box->hi[0] > box->lo[0] && box->hi[1] > box->lo[1] && box->hi[2] > box->lo[2];
    if (box->periodic) {
        for (int a = 0; a < 3; ++a) { lo[a] = 0.0; hi[a] = box->L[a]; }
    } else if (given) {
        for (int a = 0; a < 3; ++a) { lo[a] = box->lo[a]; hi[a] = box->hi[a]; }
    } else {
        pc_status s = pc_aabb(xyz, n, stream, lo, hi);
        if (s != PC_OK) return s;
    }
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) vol *= std::max(hi[a] - lo[a], 1e-300);
    const double c0 = pc_suggest_cell_size(n, vol, reach, b->mode);
    *out = o;
    out->cell_size = c0;
    if (out->ipt == 0) out->ipt = 2;
    if (n < 2) return PC_OK;

    int dev = 0, sms = 1;
    PC_CUDA(cudaGetDevice(&dev));
    PC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int nbins = b->n_a * (b->mode == PC_BIN_S ? 1 : b->n_b);
    DevBuf dc, dw;
    PC_CUDA(::pc::alloc_dev(&dc.p, sizeof(long long) * nbins));
    if (w) PC_CUDA(::pc::alloc_dev(&dw.p, sizeof(double) * nbins));

    // Sample every S-th point block.  S starts where every persistent CTA
    // still gets about four blocks, and grows (after one calibration run at
    // the model's cell side) until a trial takes about TRIAL_MS, but never so
    // far that a CTA gets fewer than two blocks.
    const double ctas = 5.0 * sms;
    const double blocks_est = std::max(1.0, (double)n / (NT * 4));
    const int S_min = std::max(1, (int)(blocks_est / (4.0 * ctas)));
    const int S_max = std::max(S_min, (int)(blocks_est / (2.0 * ctas)));
    const float TRIAL_MS = 40.f;
    int S = S_min;
    {
        pc_opts oc = o;
        oc.cell_size = c0;
        pc_grid *g = nullptr;
        pc_status s = pc_build_grid(xyz, w, w_is_f32, n, box, reach, &oc, stream, &g);
        if (s != PC_OK) return s;
        oc.ipt = 2;
        oc.shard_index = 0;
        oc.shard_count = S;
        pc_stats sts;
        s = pc_count_auto(g, b, &oc, stream, (long long *)dc.p, (double *)dw.p, &sts);
        pc_free_grid(g);
        if (s != PC_OK) return s;
        const float ms = sts.ms_pairs + sts.ms_rescue;
        if (ms > TRIAL_MS)
            S = std::min(S_max, (int)std::min(1e9, ceil(S * (double)ms / TRIAL_MS)));
    }

    const bool fp32 = o.prec == PC_PREC_F32_RESCUE;
    const bool fixed_priv = o.priv == 1 || o.priv == 2;
    if (!fixed_priv) out->priv = 0;
    float best_ms = INFINITY;
    int nt = 0;
    // one timed trial: the sampled pair and rescue kernels of grid g
    auto trial = [&](pc_grid *g, const pc_opts &oc, float &ms) -> pc_status {
        pc_opts ot = oc;
        ot.shard_index = 0;
        ot.shard_count = S;
        ms = INFINITY;
        pc_status s = PC_OK;
        for (int rep = 0; rep < 2 && s == PC_OK; ++rep) {
            pc_stats sts;
            s = pc_count_auto(g, b, &ot, stream, (long long *)dc.p, (double *)dw.p, &sts);
            if (s == PC_OK) ms = std::min(ms, sts.ms_pairs + sts.ms_rescue);
            if (ms > 4.f * TRIAL_MS) break;   // long trials: one repetition
        }
        return s;
    };
    auto record = [&](double c, int ipt, float ms) {
        if (nt < max_trials) trials[nt] = pc_tune_trial{c, ipt, fixed_priv ? o.priv : 0, ms};
        ++nt;
        if (ms < best_ms) {
            best_ms = ms;
            out->cell_size = c;
            out->ipt = ipt;
        }
    };
    // 1. i-points per thread at the model's cell side
    int ipt_best = 2;
    {
        pc_opts oc = o;
        oc.cell_size = c0;
        pc_grid *g = nullptr;
        pc_status s = pc_build_grid(xyz, w, w_is_f32, n, box, reach, &oc, stream, &g);
        if (s != PC_OK) return s;
        float ms2 = INFINITY, ms4 = INFINITY;
        oc.ipt = 2;
        s = trial(g, oc, ms2);
        if (s == PC_OK && fp32) {   // the FP64 kernel holds one point per thread
            oc.ipt = 4;
            s = trial(g, oc, ms4);
        }
        pc_free_grid(g);
        if (s != PC_OK) return s;
        record(c0, 2, ms2);
        if (fp32) record(c0, 4, ms4);
        ipt_best = ms4 < ms2 ? 4 : 2;
    }
    // 2. cell sides in quarter-octave steps from 0.7 to 2 times the model's
    //    (distinct grids only; the model's own side was timed above)
    std::vector<long long> seen;
    {
        long long ng[3];
        grid_dims(box, lo, hi, c0, ng);
        seen.push_back((ng[0] * 65537LL + ng[1]) * 65537LL + ng[2]);
    }
    for (int k = -2; k <= 4; ++k) {
        const double c = c0 * exp2(0.25 * k);
        if (k == 0 || c > 2.0 * reach || c < reach / 16.0) continue;
        long long ng[3];
        grid_dims(box, lo, hi, c, ng);
        const long long key = (ng[0] * 65537LL + ng[1]) * 65537LL + ng[2];
        if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
        seen.push_back(key);
        pc_opts oc = o;
        oc.cell_size = c;
        oc.ipt = ipt_best;
        pc_grid *g = nullptr;
        pc_status s = pc_build_grid(xyz, w, w_is_f32, n, box, reach, &oc, stream, &g);
        if (s == PC_EOVERFLOW) continue;   // too many cells at this side
        if (s != PC_OK) return s;
        float ms = INFINITY;
        s = trial(g, oc, ms);
        pc_free_grid(g);
        if (s != PC_OK) return s;
        record(c, ipt_best, ms);
    }
    // histogram replication (automatic vs one copy per warp) at the best cell
    // side and i-tile, unless the caller fixed it
    if (!fixed_priv && std::isfinite(best_ms)) {
        pc_opts oc = *out;
        pc_grid *g = nullptr;
        pc_status s = pc_build_grid(xyz, w, w_is_f32, n, box, reach, &oc, stream, &g);
        if (s != PC_OK) return s;
        pc_opts ot = oc;
        ot.priv = 1;
        ot.shard_index = 0;
        ot.shard_count = S;
        float ms = INFINITY;
        for (int rep = 0; rep < 2 && s == PC_OK; ++rep) {
            pc_stats sts;
            s = pc_count_auto(g, b, &ot, stream, (long long *)dc.p, (double *)dw.p, &sts);
            if (s == PC_OK) ms = std::min(ms, sts.ms_pairs + sts.ms_rescue);
            if (ms > 4.f * TRIAL_MS) break;
        }
        pc_free_grid(g);
        if (s != PC_OK) return s;
        if (nt < max_trials) trials[nt] = pc_tune_trial{out->cell_size, out->ipt, 1, ms};
        ++nt;
        if (ms < best_ms) {
            best_ms = ms;
            out->priv = 1;
        }
    }
    // near-edge pairs evaluated inside the pair kernel (no queue, no rescue
    // kernel: the binary64 work interleaves with the FP32 pairs of other
    // warps) at the best options, unless the caller fixed the queue size
    if (fp32 && o.rescue_capacity == 0 && std::isfinite(best_ms)) {
        pc_opts oc = *out;
        pc_grid *g = nullptr;
        pc_status s = pc_build_grid(xyz, w, w_is_f32, n, box, reach, &oc, stream, &g);
        if (s != PC_OK) return s;
        pc_opts ot = oc;
        ot.rescue_capacity = -1;
        ot.shard_index = 0;
        ot.shard_count = S;
        float ms = INFINITY;
        for (int rep = 0; rep < 2 && s == PC_OK; ++rep) {
            pc_stats sts;
            s = pc_count_auto(g, b, &ot, stream, (long long *)dc.p, (double *)dw.p, &sts);
            if (s == PC_OK) ms = std::min(ms, sts.ms_pairs + sts.ms_rescue);
            if (ms > 4.f * TRIAL_MS) break;
        }
        pc_free_grid(g);
        if (s != PC_OK) return s;
        if (nt < max_trials) trials[nt] = pc_tune_trial{out->cell_size, out->ipt, out->priv, ms};
        ++nt;
        if (ms < best_ms) {
            best_ms = ms;
            out->rescue_capacity = -1;
        }
    }
    if (n_trials) *n_trials = std::min(nt, max_trials);
    PC_CUDA(cudaStreamSynchronize(st));
    return PC_OK;
}

// Measured choice of the k-d tree path's options: the list level (through
// the list-node capacity of pc_build_tree) and the i-points per thread,
// timed like pc_tune on every S-th point block of the catalogue's auto count.
// (pc_tune_trial.cell_size carries the list-node capacity tried.)
extern "C" pc_status pc_tune_tree(const double *xyz, const void *w, int w_is_f32, long long n,
                                  const pc_box *box, const pc_bins *b, int n_leaf,
                                  const pc_opts *base, void *stream, pc_opts *out,
                                  int *list_cap, pc_tune_trial *trials, int max_trials,
                                  int *n_trials) {
    if (n_trials) *n_trials = 0;
    if (!box || !b || !out || !list_cap || n < 0 || (n > 0 && !xyz) || max_trials < 0 ||
        (max_trials > 0 && !trials))
        return fail(PC_EINVAL, "pc_tune_tree: bad arguments");
    if (b->n_a < 1 || !b->edges_a || (b->mode != PC_BIN_S && (b->n_b < 1 || !b->edges_b)))
        return fail(PC_EINVAL, "pc_tune_tree: bad bins");
    pc_opts o;
    memset(&o, 0, sizeof(o));
    o.priv = -1;
    if (base) o = *base;
    *out = o;
    out->ipt = 2;
    *list_cap = 0;
    if (n < 2) return PC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    PC_CUDA(cudaGetDevice(&dev));
    PC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int nbins = b->n_a * (b->mode == PC_BIN_S ? 1 : b->n_b);
    DevBuf dc, dw;
    PC_CUDA(::pc::alloc_dev(&dc.p, sizeof(long long) * nbins));
    if (w) PC_CUDA(::pc::alloc_dev(&dw.p, sizeof(double) * nbins));

    const double ctas = 5.0 * sms;
    const double blocks_est = std::max(1.0, (double)n / (NT * 4));
    const int S_min = std::max(1, (int)(blocks_est / (4.0 * ctas)));
    const int S_max = std::max(S_min, (int)(blocks_est / (2.0 * ctas)));
    const float TRIAL_MS = 40.f;
    int S = S_min;
    float best_ms = INFINITY;
    int nt = 0;
    auto run = [&](pc_tree *t, int ipt, float &ms) -> pc_status {
        pc_opts ot = o;
        ot.ipt = ipt;
        ot.shard_index = 0;
        ot.shard_count = S;
        ms = INFINITY;
        pc_status s = PC_OK;
        for (int rep = 0; rep < 2 && s == PC_OK; ++rep) {
            pc_stats sts;
            s = pc_count_tree(t, nullptr, b, &ot, stream, (long long *)dc.p, (double *)dw.p, &sts);
            if (s == PC_OK) ms = std::min(ms, sts.ms_pairs + sts.ms_rescue);
            if (ms > 4.f * TRIAL_MS) break;
        }
        return s;
    };
    // list-node capacities: automatic, then 512 .. 4096 (distinct levels only);
    // another option replaces the automatic level with 2 i-points only when
    // it is faster by more than the trials' run-to-run spread (3 %)
    float ms_default = INFINITY;
    std::vector<int> seen_levels;
    const int caps[] = {0, 512, 1024, 2048, 4096};
    bool calibrated = false;
    for (int cap : caps) {
        pc_tree *t = nullptr;
        pc_status s = pc_build_tree(xyz, w, w_is_f32, n, box, n_leaf, cap, stream, &t);
        if (s != PC_OK) return s;
        int depth = 0, lev = 0;
        pc_tree_info(t, nullptr, &depth, &lev, nullptr);
        if (std::find(seen_levels.begin(), seen_levels.end(), lev) != seen_levels.end()) {
            pc_free_tree(t);
            continue;
        }
        seen_levels.push_back(lev);
        if (!calibrated) {   // sampling stride from one run at the automatic level
            float ms = INFINITY;
            s = run(t, 2, ms);
            if (s != PC_OK) { pc_free_tree(t); return s; }
            if (ms > TRIAL_MS)
                S = std::min(S_max, (int)std::min(1e9, ceil(S * (double)ms / TRIAL_MS)));
            calibrated = true;
        }
        for (int ipt : {2, 4}) {
            float ms = INFINITY;
            s = run(t, ipt, ms);
            if (s != PC_OK) { pc_free_tree(t); return s; }
            if (nt < max_trials) trials[nt] = pc_tune_trial{(double)cap, ipt, o.priv, ms};
            ++nt;
            if (cap == 0 && ipt == 2) ms_default = ms;
            if (ms < best_ms) {
                best_ms = ms;
                out->ipt = ipt;
                *list_cap = cap;
            }
        }
        pc_free_tree(t);
    }
    if (std::isfinite(ms_default) && best_ms > 0.97f * ms_default) {
        out->ipt = 2;
        *list_cap = 0;
        best_ms = ms_default;
    }
    // near-edge pairs evaluated inside the pair kernel, at the chosen options
    if (o.rescue_capacity == 0 && o.prec == PC_PREC_F32_RESCUE && std::isfinite(best_ms)) {
        pc_tree *t = nullptr;
        pc_status s = pc_build_tree(xyz, w, w_is_f32, n, box, n_leaf, *list_cap, stream, &t);
        if (s != PC_OK) return s;
        pc_opts keep = o;
        o.rescue_capacity = -1;
        float ms = INFINITY;
        s = run(t, out->ipt, ms);
        o = keep;
        pc_free_tree(t);
        if (s != PC_OK) return s;
        if (nt < max_trials) trials[nt] = pc_tune_trial{(double)*list_cap, out->ipt, -1, ms};
        ++nt;
        if (ms < best_ms) out->rescue_capacity = -1;
    }
    if (n_trials) *n_trials = std::min(nt, max_trials);
    PC_CUDA(cudaStreamSynchronize(st));
    return PC_OK;
}
