// Host side of libpaircount: argument checks, the counting plan (stencil,
// lookup tables, FP32 error bands), device workspace, and the count entry
// points pc_count_auto / pc_count_cross / pc_count_batch.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <atomic>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "pc_host.hpp"

namespace pc {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

pc_status fail(pc_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

pc_status cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    set_error(m);
    if (e == cudaErrorMemoryAllocation) return PC_ENOMEM;
    return PC_ECUDA;
}

static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n); }
long long launch_count() { return g_launches.load(); }

static std::atomic<long long> g_allocs{0};
void note_alloc() { g_allocs.fetch_add(1); }
long long alloc_count() { return g_allocs.load(); }

std::mutex &api_mutex() {
    static std::mutex m;
    return m;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// device workspace (grown on demand, reused across calls)
// ---------------------------------------------------------------------------
struct Buf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max(bytes, cap * 3 / 2);
        cudaError_t e = ::pc::alloc_dev(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            want = bytes;
            e = ::pc::alloc_dev(&p, want);
        }
        if (e == cudaSuccess) cap = want;
        return e;
    }
};

struct Workspace {
    Buf hist, whist, counters, scalars, queue, blocks, tmp_cnt, tmp_off, tmp_tot, tasks, stencil, lut,
        ea, eb, fold;
};

// Fold mode (PairParams::wfold): each of the launch's `grid` CTAs gets its
// own 128-bit sums per bin in the workspace.
static pc_status attach_fold(Workspace &W, PairParams &p, int grid) {
    if (!p.wfold) return PC_OK;
    PC_CUDA(W.fold.ensure(sizeof(unsigned long long) * 2 * (size_t)p.nbins *
                          (size_t)std::max(grid, 1)));
    p.wfold_buf = (unsigned long long *)W.fold.p;
    return PC_OK;
}

static Workspace &workspace(int dev) {
    static std::map<int, Workspace> ws;
    return ws[dev];
}

// ---------------------------------------------------------------------------
// plan: bins, error bands, lookup tables, stencil
// ---------------------------------------------------------------------------
struct Plan {
    int mode = 0, los = 0, na = 0, nb = 1, nbins = 0;
    std::vector<double> ea, eb;   // edges
    std::vector<double> Ea, Eb;   // squared edges
    double reff = 0, rcut = 0;
    float eps_a = 0, eps_b = 0, mu_A = 0, mu_B = 0, mu_W = 0;
    std::vector<float2> lut;
    LutDesc la{0, 0, 0.f}, lb{0, 0, 0.f};
    std::vector<int4> stencil;
    float r2cut = 0;
    int fp32_ok = 1;              // error bands usable (else use the FP64 path)
    std::string fp32_why;
    // evenly spaced edges: bins by floor (see PairParams::lin*)
    int lin = 0;
    float lin_invA = 0, lin_offA = 0, lin_thrA = 0, lin_nB = 0, lin_mA = 0, lin_cB = 0;
    int lin_norange = 0, lin_log = 0;
    float lin_invB2 = 0, lin_thrB = 0;
    float lin_offA1 = 0;         // lin_offA + 1, rounded once
    float lin_mS = 0;
};

static bool edges_ok(const double *e, int n, bool zero_one) {
    if (n < 1 || !e) return false;
    for (int k = 0; k <= n; ++k)
        if (!(e[k] >= 0.0) || !isfinite(e[k])) return false;
    for (int k = 0; k < n; ++k)
        if (!(e[k + 1] > e[k])) return false;
    if (zero_one && !(e[0] == 0.0 && e[n] == 1.0)) return false;
    return true;
}

static const double U32 = 5.9604644775390625e-08;   // 2^-24

static float bits_f(int v) {
    float f;
    memcpy(&f, &v, sizeof(f));
    return f;
}

// Lookup table over [0, V): T cells of width V/T, each holding the single
// decision edge within `win` of the cell (or +inf if none, NaN if several)
// and the bin index just below it.  `closed_mu`: the quantity is mu, whose
// first and last edges (0 and 1) are not decisions.
static void build_lut(const std::vector<double> &e, bool closed_mu, double V, double win,
                      std::vector<float2> &out, LutDesc &d) {
    const int n = (int)e.size() - 1;
    std::vector<double> dec;      // decision edges
    std::vector<int> below;       // bin index just below each decision edge
    for (int m = 0; m <= n; ++m) {
        if (closed_mu && (m == 0 || m == n)) continue;
        if (!closed_mu && m == 0 && e[0] == 0.0) continue;   // v >= 0 always holds
        dec.push_back(e[m]);
        below.push_back(m - 1);
    }
    auto bin_of = [&](double v) {   // bin of a value away from every edge
        if (closed_mu) {
            int j = 0;
            for (int m = 1; m < n; ++m) if (v >= e[m]) j = m;
            return j;
        }
        int k = -1;
        for (int m = 0; m <= n; ++m) if (v >= e[m]) k = m;
        return k;   // -1 below e[0], n at or above e[n]
    };
    // smallest table (power of two) whose windows hold at most one edge each
    int T = 16;
    for (; T < MAX_LUT; T *= 2) {
        double w = V / T;
        bool clash = false;
        for (size_t m = 1; m < dec.size() && !clash; ++m)
            if (dec[m] - dec[m - 1] <= w + 2.0 * win) clash = true;
        if (!clash) break;
    }
    float inv_w = (float)(T / V);
    d.off = (int)out.size();
    d.T = T;
    d.inv_w = inv_w;
    const double cw = 1.0 / (double)inv_w;   // actual cell width in value units
    for (int t = 0; t <= T + 1; ++t) {
        float2 ent;
        if (t == T + 1) {   // NaN / inf inputs land here: always rescue
            ent.x = bits_f(0x7fc00000);
            ent.y = bits_f(0);
            out.push_back(ent);
            continue;
        }
        double lo = t * cw - win, hi = (t + 1) * cw + win;
        int cnt = 0, which = -1;
        for (size_t m = 0; m < dec.size(); ++m)
            if (dec[m] >= lo && dec[m] <= hi) { ++cnt; which = (int)m; }
        if (cnt == 0) {
            ent.x = INFINITY;
            int k = bin_of(std::max(0.0, t * cw + 0.5 * cw));
            ent.y = bits_f(k);
        } else if (cnt == 1) {
            ent.x = (float)dec[which];
            ent.y = bits_f(below[which]);
        } else {
            ent.x = bits_f(0x7fc00000);
            ent.y = bits_f(0);
        }
        out.push_back(ent);
    }
}

// Stencil rows (dy, dz, xlo, xhi) of cells whose minimum distance to the
// reference cell is below r (half shell for auto counts, Sect. 3.1).
static void build_stencil(const Geom &g, double r, bool half, std::vector<int4> &rows,
                          int kmax[3]) {
    rows.clear();
    const double slack = 1e-9 * std::max({g.c[0], g.c[1], g.c[2], fabs(g.lo[0]) + g.L[0],
                                           fabs(g.lo[1]) + g.L[1], fabs(g.lo[2]) + g.L[2]});
    auto md = [&](int k, int a) {
        double v = std::max(std::abs(k) - 1, 0) * g.c[a] - 2.0 * slack;
        return v > 0 ? v : 0.0;
    };
    int ky = (int)ceil(r / g.c[1]) + 1, kz = (int)ceil(r / g.c[2]) + 1;
    kmax[0] = kmax[1] = kmax[2] = 0;
    double r2 = r * r;
    for (int dz = -kz; dz <= kz; ++dz) {
        for (int dy = -ky; dy <= ky; ++dy) {
            double m2 = md(dy, 1) * md(dy, 1) + md(dz, 2) * md(dz, 2);
            if (m2 >= r2) continue;
            int rx = 0;
            while (true) {
                double mx = md(rx + 1, 0);
                if (mx * mx + m2 < r2) ++rx; else break;
            }
            int xlo = -rx, xhi = rx;
            if (half) {
                // Sect. 3.1 duplicate removal: of every row pair (dy, dz),
                // (-dy, -dz) exactly one is visited.  The kept member alternates
                // with the parity of dy + dz (the parity is the same for both),
                // so the visited half reaches equally far up and down: every
                // warp's i-points then see the same volume wherever they sit in
                // the cell, and the warps of a CTA stay balanced.
                if (dz == 0 && dy == 0) {
                    if (rx < 1) continue;
                    xlo = 1;
                } else {
                    const bool upper = dz > 0 || (dz == 0 && dy > 0);
                    if (upper == (((dy + dz) & 1) != 0)) continue;
                }
            }
            rows.push_back(make_int4(dy, dz, xlo, xhi));
            kmax[0] = std::max(kmax[0], rx);
            kmax[1] = std::max(kmax[1], std::abs(dy));
            kmax[2] = std::max(kmax[2], std::abs(dz));
        }
    }
}

static pc_status make_plan(const pc_bins *b, const Geom &g, const double *pts_lo,
                           const double *pts_hi, double rmin, bool half, Plan &P,
                           bool with_stencil = true) {
    if (!b) return fail(PC_EINVAL, "bins: NULL");
    if (b->mode < 0 || b->mode > 2) return fail(PC_EINVAL, "bins: unknown mode");
    if (b->los < 0 || b->los > 1) return fail(PC_EINVAL, "bins: unknown line of sight");
    P.mode = b->mode;
    P.los = (b->mode == PC_BIN_S) ? PC_LOS_Z : b->los;
    if (!edges_ok(b->edges_a, b->n_a, false))
        return fail(PC_EINVAL, "bins: edges_a must be finite, >= 0 and strictly increasing");
    P.na = b->n_a;
    P.ea.assign(b->edges_a, b->edges_a + b->n_a + 1);
    if (P.mode == PC_BIN_S) {
        P.nb = 1;
        P.eb = {0.0, 1.0};
    } else {
        if (!edges_ok(b->edges_b, b->n_b, P.mode == PC_BIN_SMU))
            return fail(PC_EINVAL, P.mode == PC_BIN_SMU
                                       ? "bins: mu edges must increase strictly from 0 to 1"
                                       : "bins: pi edges must be finite, >= 0 and increasing");
        P.nb = b->n_b;
        P.eb.assign(b->edges_b, b->edges_b + b->n_b + 1);
    }
    if ((long long)P.na * P.nb > (1LL << 26)) return fail(PC_EOVERFLOW, "bins: too many bins");
    P.nbins = P.na * P.nb;
    if (g.periodic && P.los == PC_LOS_MIDPOINT)
        return fail(PC_EINVAL, "bins: the midpoint line of sight needs a non-periodic box");
    P.Ea.resize(P.na + 1);
    P.Eb.resize(P.nb + 1);
    for (int k = 0; k <= P.na; ++k) P.Ea[k] = P.ea[k] * P.ea[k];
    for (int k = 0; k <= P.nb; ++k) P.Eb[k] = P.eb[k] * P.eb[k];
    P.reff = (P.mode == PC_BIN_SIGPI) ? sqrt(P.ea[P.na] * P.ea[P.na] + P.eb[P.nb] * P.eb[P.nb])
                                      : P.ea[P.na];

    // ---- FP32 error bands (derivation in the design notes) -----------------
    const double u = U32;
    const double c = std::max({g.c[0], g.c[1], g.c[2]});
    double X = 0.0, Lm = 0.0;
    for (int a = 0; a < 3; ++a) {
        X = std::max({X, fabs(pts_lo[a]), fabs(pts_hi[a])});
        Lm = std::max(Lm, g.L[a]);
    }
    const double R0 = P.reff;
    const double tiny = ldexp(X + Lm + R0, -48);
    // separation length s (and sigma along z) and the z component
    double Rb = R0 * (1.0 + 1e-6) + 1e-6 * c;
    double eps_s = 2.0 * u * (4.4 * c + 10.5 * Rb) + tiny;
    double eps_z = 2.0 * u * (2.5 * c + 4.0 * Rb) + tiny;
    double eps_sig = 2.0 * u * (3.6 * c + 11.5 * Rb) + ldexp(Rb, -25) + tiny;
    double muA = 2.0 * (6.9 * u * c) + tiny, muB = 2.0 * 21.0 * u + ldexp(1.0, -48);
    if (P.los == PC_LOS_MIDPOINT) {
        // distance of the nearest point to the observer bounds |x_i + x_j|:
        // the larger of the bounding box's distance and the points' own
        // smallest radius (a shell is far from the observer although its
        // bounding box may come close)
        double dmin2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double d = 0.0;
            if (pts_lo[a] > 0.0) d = pts_lo[a];
            else if (pts_hi[a] < 0.0) d = -pts_hi[a];
            dmin2 += d * d;
        }
        const double dmin = std::max(sqrt(dmin2) * (1.0 - 1e-12), rmin);
        double lmin = 2.0 * dmin - Rb;
        double dl = u * (5.5 * X + 4.4 * c + 6.2 * Rb);
        if (lmin > 4.0 * Rb) {
            double em = 2.0 * (u * (4.4 * c + 17.5 * Rb) + 2.0 * Rb * dl / lmin) +
                        ldexp(Rb, -25) + tiny;
            eps_sig = em;
            eps_z = em;
            muA = em + eps_s;
            muB = 2.0 * 8.0 * u + ldexp(1.0, -48);
        } else {
            P.fp32_ok = 0;
            P.fp32_why = "observer too close to the points for the FP32 midpoint bound";
        }
    }
    P.rcut = R0 + std::max({eps_s, eps_z, eps_sig}) * 2.0;
    {
        double r2 = P.rcut * P.rcut * (1.0 + 8.0 * u);
        P.r2cut = nextafterf((float)r2, INFINITY);
    }
    // ---- lookup tables ------------------------------------------------------
    const double V = P.rcut * (1.0 + 1e-5) + 1e-30;
    P.lut.clear();
    if (P.mode == PC_BIN_S) {
        P.eps_a = (float)(eps_s * (1.0 + 1e-6));
        build_lut(P.ea, false, V, 2.0 * eps_s, P.lut, P.la);
        P.lb = P.la;
    } else if (P.mode == PC_BIN_SMU) {
        P.eps_a = (float)(eps_s * (1.0 + 1e-6));
        P.mu_A = (float)(muA * (1.0 + 1e-6));
        P.mu_B = (float)(muB * (1.0 + 1e-6));
        build_lut(P.ea, false, V, 2.0 * eps_s, P.lut, P.la);
        // mu window: the band of a pair must fit in it (else always rescue)
        double minGap = 1.0;
        for (int k = 0; k < P.nb; ++k) minGap = std::min(minGap, P.eb[k + 1] - P.eb[k]);
        double wmu = std::min(1e-3, 0.2 * minGap);
        P.mu_W = (float)wmu;
        build_lut(P.eb, true, 1.0 + 1e-3, wmu, P.lut, P.lb);
    } else {
        P.eps_a = (float)(eps_sig * (1.0 + 1e-6));
        P.eps_b = (float)(eps_z * (1.0 + 1e-6));
        build_lut(P.ea, false, V, 2.0 * eps_sig, P.lut, P.la);
        build_lut(P.eb, false, V, 2.0 * eps_z, P.lut, P.lb);
    }
    // ---- evenly spaced edges: floor-based bins ------------------------------
    // s (and mu along z): bin = floor(t), t = (s - e0) / D, with the band
    // moved into t units plus the rounding of t itself (scaling factor and
    // offset rounded to FP32, one FMA) and the edges' distance from exact
    // even spacing.
    {
        const double e0 = P.ea[0], D = (P.ea[P.na] - P.ea[0]) / P.na;
        double dev = 0.0;
        for (int k = 0; k <= P.na; ++k) dev = std::max(dev, fabs(P.ea[k] - (e0 + k * D)));
        bool lin_s = dev <= 1e-9 * D;
        bool lin_mu = true;
        double devm = 0.0;
        if (P.mode == PC_BIN_SMU) {
            for (int k = 0; k <= P.nb; ++k) devm = std::max(devm, fabs(P.eb[k] - (double)k / P.nb));
            lin_mu = (P.los == PC_LOS_Z) && devm <= 1e-12;
        }
        bool mode_ok = P.mode == PC_BIN_S || (P.mode == PC_BIN_SMU && P.los == PC_LOS_Z);
        if (lin_s && lin_mu && mode_ok && (P.rcut - e0) / D < 4.0e6) {
            double ts_max = (P.rcut - e0) / D + 1.0;
            double eps_t = (eps_s + dev) / D + 4.0 * u * (ts_max + fabs(e0) / D);
            if (eps_t < 0.25) {
                P.lin = 1;
                P.lin_invA = (float)(1.0 / D);
                P.lin_offA = (float)(-e0 / D);
                P.lin_offA1 = (float)(1.0 - e0 / D);
                P.lin_thrA = nextafterf((float)(0.5 - eps_t), 0.0f);
                // e_0 = 0: t_s = s / D >= 0; and every candidate has t_s below
                // n_a + 1/2 (plus rounding), so floor(t_s) <= n_a
                P.lin_norange = (e0 == 0.0 && ts_max - 1.0 <= P.na + 0.5) ? 1 : 0;
                if (P.mode == PC_BIN_SMU) {
                    // t_mu = mu n_mu (1 - 2^-21): below n_mu for every pair (mu
                    // = |dz| rsqrt(s^2) exceeds 1 by at most ~3e-7), so mu = 1
                    // lands in the last bin without a clamp; the scale's shift
                    // of up to 2^-21 n_mu joins the band
                    const double nb = P.nb;
                    P.lin_nB = nextafterf((float)(nb * (1.0 - ldexp(1.0, -21))), 0.0f);
                    P.lin_mA = (float)(muA * nb * (1.0 + 1e-6));
                    double cB = 0.5 - (muB + 4.0 * u + devm + ldexp(1.0, -21)) * nb;
                    P.lin_cB = nextafterf((float)cB, 0.0f);
                    if (!(cB > 0.25)) P.lin = 0;
                }
            }
        }
    }
    // ---- logarithmic s edges: floor of a scaled base-2 logarithm -----------
    // e_k = e_0 q^k: bin = floor(t), t = log_q(s / e_0) = A log2(s^2) + B with
    // A = 1 / (2 log2 q), B = -log2(e_0) / log2 q (Sect. 3.2's log mapping).
    // Band in t units (each term times 2 below, like the linear case):
    //  - the separation vector's error u (4.33 c + 3 s) + 2^-51 X (c the cell
    //    side) is relative in log2(s^2): 2 (4.33 u c + 2^-51 X) / (s ln 2) plus
    //    6u / ln 2, and the three roundings of s^2 add 3u / ln 2 -- the 1/s
    //    part is applied per pair through rsqrt(s^2);
    //  - the hardware base-2 logarithm errs by at most 2^-21 max(1, |log2 x|)
    //    (twice the largest error over every positive normal binary32 input,
    //    measured exhaustively on the device by the test suite);
    //  - A, B rounded to binary32 and the FMA add u (A |L| + |B| + |t|);
    //  - the edges' distance from an exact geometric sequence (in t units),
    //    and the oracle's binary64 roundings (2^-45 A).
    if (!P.lin && P.ea[0] > 0.0) {
        const double e0 = P.ea[0], lq = log2(P.ea[P.na] / e0) / P.na;
        bool lin_mu = true;
        double devm = 0.0;
        if (P.mode == PC_BIN_SMU) {
            for (int k = 0; k <= P.nb; ++k) devm = std::max(devm, fabs(P.eb[k] - (double)k / P.nb));
            lin_mu = (P.los == PC_LOS_Z) && devm <= 1e-12;
        }
        bool mode_ok = P.mode == PC_BIN_S || (P.mode == PC_BIN_SMU && P.los == PC_LOS_Z);
        double dev = 0.0;
        for (int k = 0; k <= P.na; ++k) dev = std::max(dev, fabs(log2(P.ea[k] / e0) / lq - k));
        if (mode_ok && lin_mu && lq > 0.0 && dev <= 1e-6 && P.na < (1 << 20)) {
            const double ln2 = log(2.0), A = 1.0 / (2.0 * lq), B = -log2(e0) / lq;
            const double Lmax = std::max(fabs(log2(P.rcut * P.rcut)), fabs(log2(0.25 * e0 * e0)));
            const double tmax = A * Lmax + fabs(B) + 1.0;
            const double C1 = A * 2.0 * (4.4 * u * c + ldexp(X + Lm + R0, -51)) / ln2 * 1.01;
            const double C0 = A * 9.0 * u / ln2 * 1.01 + A * ldexp(1.0, -21) * std::max(1.0, Lmax) +
                              u * (A * Lmax + fabs(B) + tmax) * 2.0 + dev + A * ldexp(1.0, -45);
            if (2.0 * C0 < 0.25) {
                P.lin = 1;
                P.lin_log = 1;
                P.lin_invA = (float)A;
                P.lin_offA = (float)B;
                P.lin_offA1 = (float)(B + 1.0);
                P.lin_thrA = nextafterf((float)(0.5 - 2.0 * C0), 0.0f);
                // rsqrt(s^2) >= (1 - 2^-22) / s: scale the 1/s term up to cover it
                P.lin_mS = nextafterf((float)(2.0 * C1 * (1.0 + 1e-6)), INFINITY);
                P.lin_norange = 0;
                if (P.mode == PC_BIN_SMU) {
                    const double nb = P.nb;   // mu scale and band as for linear s bins
                    P.lin_nB = nextafterf((float)(nb * (1.0 - ldexp(1.0, -21))), 0.0f);
                    P.lin_mA = (float)(muA * nb * (1.0 + 1e-6));
                    double cB = 0.5 - (muB + 4.0 * u + devm + ldexp(1.0, -21)) * nb;
                    P.lin_cB = nextafterf((float)cB, 0.0f);
                    if (!(cB > 0.25)) P.lin = P.lin_log = 0;
                }
            }
        }
    }
    // ---- (sigma, pi) with evenly spaced edges from 0: floors of both ------
    // t_sigma = sigma / D_a, t_pi = pi / D_b, sigma and pi formed as on the
    // table path, so their bands eps_sig and eps_z apply (in t units), plus
    // the rounding of the scale and product (2u t) and the edges' distance
    // from even spacing.
    if (!P.lin && P.mode == PC_BIN_SIGPI && P.fp32_ok && P.ea[0] == 0.0 && P.eb[0] == 0.0) {
        const double Da = P.ea[P.na] / P.na, Db = P.eb[P.nb] / P.nb;
        double deva = 0.0, devb = 0.0;
        for (int k = 0; k <= P.na; ++k) deva = std::max(deva, fabs(P.ea[k] - k * Da));
        for (int k = 0; k <= P.nb; ++k) devb = std::max(devb, fabs(P.eb[k] - k * Db));
        const double tma = P.rcut / Da + 1.0, tmb = P.rcut / Db + 1.0;
        const double eta = (eps_sig + deva) / Da + 4.0 * u * tma;
        const double etb = (eps_z + devb) / Db + 4.0 * u * tmb;
        if (deva <= 1e-9 * Da && devb <= 1e-9 * Db && tma < 4.0e6 && tmb < 4.0e6 && eta < 0.25 &&
            etb < 0.25) {
            P.lin = 1;
            P.lin_invA = (float)(1.0 / Da);
            P.lin_offA = 0.0f;
            P.lin_offA1 = 0.0f;
            P.lin_thrA = nextafterf((float)(0.5 - eta), 0.0f);
            P.lin_invB2 = (float)(1.0 / Db);
            P.lin_thrB = nextafterf((float)(0.5 - etb), 0.0f);
            P.lin_norange = 0;
        }
    }
    // ---- stencil -------------------------------------------------------------
    int kmax[3] = {0, 0, 0};
    P.stencil.clear();
    if (with_stencil) build_stencil(g, P.rcut, half, P.stencil, kmax);
    if (g.periodic) {
        for (int a = 0; a < 3; ++a) {
            if (!(P.rcut < 0.5 * g.L[a]))
                return fail(PC_EINVAL,
                            "bins: the largest separation must stay below half the periodic box");
            if (with_stencil && 2 * kmax[a] + 1 > g.ng[a])
                return fail(PC_EINVAL,
                            "grid: cells too large for this separation in a periodic box "
                            "(neighbour cells would alias); rebuild with a smaller cell_size");
        }
    }
    return PC_OK;
}

// ---------------------------------------------------------------------------
// one counting launch over a set of tasks
// ---------------------------------------------------------------------------
// Histogram replication from pc_opts.priv: 1 = one count copy per warp,
// 2 = a single shared copy, otherwise automatic: lane copies (lane l updates
// copy l % k) as many as fit a 16 KB budget, so the lanes of a warp do not
// collide on the few bins of a small histogram.
// (weighted: binary64 weight sums share the copies and the budget; the
// integer weight records take the counts' copies outside that budget.)
static void choose_replication(int mode, int nbins, bool weighted, int &priv, int &hist_k) {
    priv = 0;
    hist_k = 1;
    if (mode == 1) { priv = 1; return; }
    if (mode == 2) return;
    const long long per_copy = (long long)nbins * (4 + (weighted ? 8 : 0));
    while (hist_k < 32 && per_copy * hist_k * 2 <= 16384) hist_k *= 2;
}

// Rows of each shared histogram copy: the bins, the discarded rows of the
// floor bins without a range test, and at least one row past the bins that
// lanes without an in-range pair update (row nbins).
static void set_hist_rows(PairParams &p, const Plan &P) {
    p.nbins_smem = P.nbins + (p.lin_norange ? (P.mode == PC_BIN_S ? 1 : P.nb) : 0);
    p.trash_row = P.nbins;
    p.nbins_smem = std::max(p.nbins_smem, P.nbins + 1);
}

// Shared-memory fallback: fewer lane copies, then no warp copies, then the
// global histogram.  Returns false when nothing is left to give up.
static bool shrink_replication(PairParams &p) {
    if (p.hist_k > 1) { p.hist_k /= 2; return true; }
    if (p.priv) { p.priv = 0; return true; }
    return false;
}

struct CountJob {
    std::vector<TaskDev> tasks;
    int nhist;
    bool is_auto;
    const pc_grid *g0 = nullptr;
    // geometry of the count (the first grid's, or the trees')
    Geom geom;
    int device = 0;
    int ncell = 0;               // cells per grid, or i-blocks of a tree count
    double plo[3] = {0, 0, 0}, phi[3] = {0, 0, 0};   // first grid's point bounds
    double cell_size = 0.0;
    bool tree = false;
    // bounds of the points of every grid involved, and a lower bound of |x|
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    double rmin = 0.0;
    bool wint_ok = true;   // every task's grids allow the integer weight path
    bool wcorr = false;    // some grid's binary64 weights add remainders
};

// Integer weight products are truncated by at most 2^(k_i + k_j - 46)
// relative, k the exponent offset of a weight below its grid's largest; the
// exponent spans of the two grids are limited so that this stays below
// 2^-34 (6e-11) per product and hence per bin.
static void job_add_wint(CountJob &J, const pc_grid *gi, const pc_grid *gj) {
    if (!gi->wint || !gj->wint ||
        (gi->wemax - gi->wemin) + (gj->wemax - gj->wemin) > WINT_MAX_SPAN)
        J.wint_ok = false;
    if (gi->wcorr || gj->wcorr) J.wcorr = true;
}

// Lower bound of |x| over the points of a grid (0 when unknown or periodic).
static double grid_rmin(const pc_grid *g) {
    if (g->g.periodic || !(g->r2min > 0.0)) return 0.0;
    return sqrt(g->r2min) * (1.0 - 1e-12);
}

// The job's geometry from its first grid.
static void job_set_grid(CountJob &J, const pc_grid *g) {
    J.g0 = g;
    J.geom = g->g;
    J.device = g->device;
    J.ncell = g->ncell;
    for (int a = 0; a < 3; ++a) {
        J.plo[a] = g->pts_lo[a];
        J.phi[a] = g->pts_hi[a];
    }
    J.cell_size = g->cell_size;
}

// Fold grid g into the job's point bounds (the first grid initialises them).
static void job_add_bounds(CountJob &J, const pc_grid *g, bool first) {
    for (int a = 0; a < 3; ++a) {
        J.lo[a] = first ? g->pts_lo[a] : std::min(J.lo[a], g->pts_lo[a]);
        J.hi[a] = first ? g->pts_hi[a] : std::max(J.hi[a], g->pts_hi[a]);
    }
    J.rmin = first ? grid_rmin(g) : std::min(J.rmin, grid_rmin(g));
}

// Everything decided on the host before any device work.
struct CountSetup {
    Plan P;
    pc_opts o;
    int prec = 0, ipt = 2, bi = 256, dev = 0, ntasks = 0, ncell = 0;
    bool weighted = false;
    int wsum = 0;   // weighted sums: 0 none, 1 binary64 products, 2 integer products,
                    // 3 integer products with binary64 remainders
    size_t nblk_cap = 0, hist_n = 0;
    unsigned long long qcap = 0;
};

// Device buffers of one count (raw pointers into a Workspace).
struct DevBufs {
    unsigned long long *hist = nullptr;
    double *whist = nullptr;
    unsigned long long *ctr = nullptr;   // [0] candidates, [1] inline rescues, [2] queue count,
                                         // [3] pairs pruned by group bounds
    int *sc = nullptr;                   // [0] work counter, [1] number of blocks
    uint3 *queue = nullptr;
    Block *blocks = nullptr;
    int *cnt = nullptr, *off = nullptr, *tot = nullptr;
    TaskDev *tasks = nullptr;
    int4 *stencil = nullptr;
    float2 *lut = nullptr;
    double *ea = nullptr, *eb = nullptr;
};

static pc_status setup_count(const CountJob &J, const pc_bins *b, const pc_opts *opt,
                             bool weighted, CountSetup &S) {
    memset(&S.o, 0, sizeof(S.o));
    S.o.priv = -1;
    if (opt) S.o = *opt;
    if (S.o.shard_count > 1 && (S.o.shard_index < 0 || S.o.shard_index >= S.o.shard_count))
        return fail(PC_EINVAL, "opts: shard_index must lie in [0, shard_count)");
    pc_status s = make_plan(b, J.geom, J.lo, J.hi, J.rmin, J.is_auto, S.P, !J.tree);
    if (s != PC_OK) return s;
    S.weighted = weighted;
    S.prec = S.o.prec;
    if (S.prec == PC_PREC_F32_RESCUE && !S.P.fp32_ok) S.prec = PC_PREC_F64;
    S.ipt = (S.o.ipt == 4) ? 4 : 2;
    if (S.prec == PC_PREC_F64) S.ipt = 1;
    S.bi = NT * S.ipt;
    S.dev = J.device;
    S.ntasks = (int)J.tasks.size();
    S.ncell = J.ncell;
    long long npts = 0;
    for (auto &t : J.tasks) npts += t.gi.n;
    S.nblk_cap = (size_t)S.ntasks * S.ncell + (size_t)(npts / S.bi) + 16;
    S.hist_n = (size_t)J.nhist * S.P.nbins;
    // rescue queue capacity: ~4e-3 of the expected in-range pairs (overflow
    // is evaluated inside the pair kernel, so this only sets the fast case)
    S.qcap = 0;
    if (S.prec == PC_PREC_F32_RESCUE) {
        if (S.o.rescue_capacity > 0) S.qcap = (unsigned long long)S.o.rescue_capacity;
        else if (S.o.rescue_capacity == 0) {
            double vol = 1.0;
            for (int a = 0; a < 3; ++a) vol *= std::max(J.phi[a] - J.plo[a], 1e-9);
            double vs = 4.0 / 3.0 * M_PI * S.P.reff * S.P.reff * S.P.reff;
            double pairs = 0.0;
            for (auto &t : J.tasks)
                pairs += 0.5 * (double)t.gi.n * (double)t.gj.n * std::min(1.0, vs / vol);
            double want = std::max(1.0e6, 4.0e-3 * pairs * (J.is_auto ? 1.0 : 2.0));
            S.qcap = (unsigned long long)std::min(want, 4.0e8);
        }
    }
    return PC_OK;
}

static pc_status ensure_bufs(Workspace &W, const CountSetup &S, DevBufs &B) {
    const size_t cells = (size_t)S.ntasks * S.ncell + 1;
    PC_CUDA(W.hist.ensure(sizeof(unsigned long long) * S.hist_n));
    if (S.weighted) PC_CUDA(W.whist.ensure(sizeof(double) * S.hist_n));
    PC_CUDA(W.counters.ensure(sizeof(unsigned long long) * 4));
    PC_CUDA(W.scalars.ensure(sizeof(int) * 4));
    PC_CUDA(W.blocks.ensure(sizeof(Block) * S.nblk_cap));
    PC_CUDA(W.tmp_cnt.ensure(sizeof(int) * cells));
    PC_CUDA(W.tmp_off.ensure(sizeof(int) * cells));
    PC_CUDA(W.tmp_tot.ensure(sizeof(int) * (cells / 4096 + 2)));
    PC_CUDA(W.tasks.ensure(sizeof(TaskDev) * S.ntasks));
    PC_CUDA(W.stencil.ensure(sizeof(int4) * std::max<size_t>(S.P.stencil.size(), 1)));
    PC_CUDA(W.lut.ensure(sizeof(float2) * std::max<size_t>(S.P.lut.size(), 1)));
    PC_CUDA(W.ea.ensure(sizeof(double) * (S.P.na + 1)));
    PC_CUDA(W.eb.ensure(sizeof(double) * (S.P.nb + 1)));
    if (S.qcap) PC_CUDA(W.queue.ensure(sizeof(uint3) * S.qcap));
    B.hist = (unsigned long long *)W.hist.p;
    B.whist = S.weighted ? (double *)W.whist.p : nullptr;
    B.ctr = (unsigned long long *)W.counters.p;
    B.sc = (int *)W.scalars.p;
    B.queue = (uint3 *)W.queue.p;
    B.blocks = (Block *)W.blocks.p;
    B.cnt = (int *)W.tmp_cnt.p;
    B.off = (int *)W.tmp_off.p;
    B.tot = (int *)W.tmp_tot.p;
    B.tasks = (TaskDev *)W.tasks.p;
    B.stencil = (int4 *)W.stencil.p;
    B.lut = (float2 *)W.lut.p;
    B.ea = (double *)W.ea.p;
    B.eb = (double *)W.eb.p;
    return PC_OK;
}

// Host-built tables of the count (tasks, stencil, lookup tables, edges).
static pc_status upload_tables(const CountJob &J, const CountSetup &S, const DevBufs &B,
                               cudaStream_t st) {
    PC_CUDA(cudaMemcpyAsync(B.tasks, J.tasks.data(), sizeof(TaskDev) * S.ntasks,
                            cudaMemcpyHostToDevice, st));
    if (!S.P.stencil.empty())
        PC_CUDA(cudaMemcpyAsync(B.stencil, S.P.stencil.data(), sizeof(int4) * S.P.stencil.size(),
                                cudaMemcpyHostToDevice, st));
    if (!S.P.lut.empty())
        PC_CUDA(cudaMemcpyAsync(B.lut, S.P.lut.data(), sizeof(float2) * S.P.lut.size(),
                                cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaMemcpyAsync(B.ea, S.P.Ea.data(), sizeof(double) * (S.P.na + 1),
                            cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaMemcpyAsync(B.eb, S.P.Eb.data(), sizeof(double) * (S.P.nb + 1),
                            cudaMemcpyHostToDevice, st));
    return PC_OK;
}

// Kernel parameters and launch shape.
static pc_status make_params(const CountJob &J, const CountSetup &S, const DevBufs &B,
                             PairParams &p, int &grid, size_t &smem) {
    const Plan &P = S.P;
    memset(static_cast<void *>(&p), 0, sizeof(p));
    p.groups = 1;
    p.tree = J.tree ? 1 : 0;
    p.tasks = B.tasks;
    p.blocks = B.blocks;
    p.nblocks = B.sc + 1;
    p.work_counter = B.sc;
    p.g = J.geom;
    p.stencil = B.stencil;
    p.nrows = (int)P.stencil.size();
    p.mode = P.mode;
    p.los = P.los;
    p.weighted = S.weighted ? 1 : 0;
    p.n_a = P.na;
    p.n_b = P.nb;
    p.nbins = P.nbins;
    p.r2cut = P.r2cut;
    p.lut = B.lut;
    p.lut_total = (int)P.lut.size();
    p.la = P.la;
    p.lb = P.lb;
    p.eps_a = P.eps_a;
    p.eps_b = P.eps_b;
    p.mu_A = P.mu_A;
    p.mu_B = P.mu_B;
    p.mu_W = P.mu_W;
    p.Ea = B.ea;
    p.Eb = B.eb;
    p.hist = B.hist;
    p.whist = B.whist;
    p.queue = B.queue;
    p.qcount = B.ctr + 2;
    p.qcap = S.qcap;
    p.counters = B.ctr;
    p.shard_count = S.o.shard_count > 1 ? S.o.shard_count : 1;
    p.shard_index = S.o.shard_count > 1 ? S.o.shard_index : 0;
    p.lin = (S.prec == PC_PREC_F32_RESCUE) ? P.lin : 0;
    p.lin_norange = p.lin ? P.lin_norange : 0;
    p.lin_log = p.lin ? P.lin_log : 0;
    p.lin_mS = P.lin_mS;
    p.lin_invB2 = P.lin_invB2;
    p.lin_thrB = P.lin_thrB;
    set_hist_rows(p, P);
    p.lin_invA = P.lin_invA;
    // the range-tested floor bins take t_s + 1 (exact floors down to t_s = -1)
    p.lin_offA = P.lin_norange ? P.lin_offA : P.lin_offA1;
    p.lin_thrA = P.lin_thrA;
    p.lin_nB = P.lin_nB;
    p.lin_mA = P.lin_mA;
    p.lin_cB = P.lin_cB;

    int dev_sms = 0, smem_optin = 0;
    PC_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, S.dev));
    PC_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, S.dev));
    const int static_smem = 256;
    const int lut_size = p.lut_total;
    // shared-memory layout for a weight path: replication, then fewer copies
    // until it fits, else the global histogram
    auto fit = [&](bool wint) {
        p.wint = wint ? 1 : 0;
        p.wcorr = (wint && J.wcorr) ? 1 : 0;
        choose_replication(S.o.priv, P.nbins, S.weighted && !wint, p.priv, p.hist_k);
        for (;;) {
            p.wint_k = p.hist_k;   // the weight records take the counts' lane copies
            p.smem_hist_ok = 1;
            // the floor-based bins need no tables (they serve only the global-
            // histogram variant)
            p.lut_total = p.lin ? 0 : lut_size;
            size_t need = (S.prec == PC_PREC_F64) ? pairs_f64_smem(p) : pairs_f32_smem(p, S.ipt);
            if (need + static_smem <= (size_t)smem_optin) break;
            if (shrink_replication(p)) continue;
            p.smem_hist_ok = 0;
            p.lut_total = lut_size;
            break;
        }
        return (S.prec == PC_PREC_F64) ? pairs_f64_smem(p) : pairs_f32_smem(p, S.ipt);
    };
    // integer weight products need floor bins, every weight packable and
    // shared histograms with one count copy per CTA; with fewer than 16 lane
    // copies (more than a few hundred bins) a copy would be flushed every few
    // hundred j-points, so its records are folded into the CTA's exact sums
    // instead (fold mode)
    const bool wint_try = S.weighted && p.lin && J.wint_ok && S.prec == PC_PREC_F32_RESCUE;
    smem = fit(wint_try);
    if (p.wint && !(p.smem_hist_ok && !p.priv)) smem = fit(false);
    p.wfold = (p.wint && p.hist_k < 16) ? 1 : 0;
    if (smem + static_smem > (size_t)smem_optin)
        return fail(PC_EUNSUPPORTED, "bins: tables do not fit in shared memory");
    int per_sm = (S.prec == PC_PREC_F64) ? pairs_f64_ctas_per_sm(p, smem)
                                         : pairs_f32_ctas_per_sm(p, S.ipt, smem);
    // A shared histogram so large that at most two CTAs of NT threads fit an
    // SM: run CTAs of four independent thread groups sharing one histogram
    // (single-histogram jobs, floor bins, binary64 or no weights, 2 i-points)
    if (S.prec == PC_PREC_F32_RESCUE && p.smem_hist_ok && p.lin && !p.wint && !p.priv &&
        J.nhist == 1 && S.ipt == 2 && per_sm <= 2 && !p.tree) {
        p.groups = 4;
        const size_t smem4 = pairs_f32_smem(p, S.ipt);
        const int per4 = (smem4 + 8192 <= (size_t)smem_optin) ? pairs_f32_ctas_per_sm(p, S.ipt, smem4) : 0;
        if (per4 >= 1) {
            smem = smem4;
            per_sm = per4;
        } else {
            p.groups = 1;
        }
    }
    if (per_sm <= 0)
        return fail(PC_ECUDA, std::string("pair kernel cannot be resident: ") + pc_last_error());
    if (S.o.grid_ctas_per_sm > 0) per_sm = std::min(per_sm, S.o.grid_ctas_per_sm);
    grid = dev_sms * per_sm;
    return PC_OK;
}

// Device work of one count, in stream order (also what a captured graph
// replays): clear, block list, pair kernel, rescue kernel.
static pc_status enqueue_count(const CountSetup &S, const DevBufs &B, const PairParams &p, int grid,
                               size_t smem, cudaStream_t st, cudaEvent_t ev_pairs,
                               cudaEvent_t ev_rescue, cudaEvent_t ev_done,
                               const std::function<cudaError_t()> &tree_blocks_fn = {}) {
    PC_CUDA(cudaMemsetAsync(B.hist, 0, sizeof(unsigned long long) * S.hist_n, st));
    if (S.weighted) PC_CUDA(cudaMemsetAsync(B.whist, 0, sizeof(double) * S.hist_n, st));
    PC_CUDA(cudaMemsetAsync(B.ctr, 0, sizeof(unsigned long long) * 4, st));
    PC_CUDA(cudaMemsetAsync(B.sc, 0, sizeof(int) * 4, st));
    if (tree_blocks_fn)   // tree counts: balanced blocks of the list nodes
        PC_CUDA(tree_blocks_fn());
    else
        PC_CUDA(make_blocks_into(B.tasks, S.ntasks, S.ncell, S.bi, p.shard_index, p.shard_count,
                                 B.blocks, B.sc + 1, B.cnt,
                                 B.off, B.tot, st));
    if (ev_pairs) PC_CUDA(cudaEventRecord(ev_pairs, st));
    cudaError_t e = (S.prec == PC_PREC_F64) ? launch_pairs_f64(p, grid, smem, st)
                                            : launch_pairs_f32(p, S.ipt, grid, smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "pair kernel launch");
    if (ev_rescue) PC_CUDA(cudaEventRecord(ev_rescue, st));
    if (S.prec == PC_PREC_F32_RESCUE && S.qcap) {
        e = launch_rescue(p, st);
        if (e != cudaSuccess) return cuda_fail(e, "rescue kernel launch");
    }
    if (ev_done) PC_CUDA(cudaEventRecord(ev_done, st));
    return PC_OK;
}

static void copy_out(void *dst, const void *src, size_t bytes, cudaStream_t st, cudaError_t &e) {
    if (!dst || e != cudaSuccess) return;
    cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    e = cudaMemcpyAsync(dst, src, bytes, k, st);
}

static void fill_stats(pc_stats *stats, const CountSetup &S, double cell_size,
                       const unsigned long long hc[4], int hblk, float ms_total, float ms_pairs,
                       float ms_rescue, long long launches) {
    if (!stats) return;
    memset(stats, 0, sizeof(*stats));
    stats->candidates = (long long)hc[0];
    stats->rescue_inline = (long long)hc[1];
    stats->pruned = (long long)hc[3];
    stats->prec = S.prec;
    stats->wsum = S.wsum;
    stats->rescued = (long long)std::min<unsigned long long>(hc[2], S.qcap) + (long long)hc[1];
    stats->blocks = hblk;
    stats->cell_size = cell_size;
    stats->ms_total = ms_total;
    stats->ms_pairs = ms_pairs;
    stats->ms_rescue = ms_rescue;
    stats->launches = (int)launches;
}

struct Events {
    cudaEvent_t e[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool on = false;
    explicit Events(bool want) : on(want) {
        if (on) for (auto &x : e) cudaEventCreate(&x);
    }
    ~Events() {
        if (on) for (auto &x : e) cudaEventDestroy(x);
    }
    float ms(int a, int b) const {
        float m = 0.f;
        if (on) cudaEventElapsedTime(&m, e[a], e[b]);
        return m;
    }
};

static pc_status run_count(const CountJob &J, const pc_bins *b, const pc_opts *opt,
                           cudaStream_t st, long long *counts, double *wcounts, pc_stats *stats) {
    CountSetup S;
    pc_status s = setup_count(J, b, opt, wcounts != nullptr, S);
    if (s != PC_OK) return s;
    DevBufs B;
    s = ensure_bufs(workspace(S.dev), S, B);
    if (s != PC_OK) return s;
    PairParams p;
    int grid = 0;
    size_t smem = 0;
    s = make_params(J, S, B, p, grid, smem);
    if (s == PC_OK) s = attach_fold(workspace(S.dev), p, grid);
    if (s != PC_OK) return s;
    S.wsum = p.wint ? (p.wcorr ? 3 : 2) : (S.weighted ? 1 : 0);
    Events ev(stats != nullptr);
    const long long launches0 = launch_count();
    if (ev.on) PC_CUDA(cudaEventRecord(ev.e[0], st));
    s = upload_tables(J, S, B, st);
    if (s != PC_OK) return s;
    s = enqueue_count(S, B, p, grid, smem, st, ev.e[1], ev.e[2], ev.e[3]);
    if (s != PC_OK) return s;
    cudaError_t e = cudaSuccess;
    copy_out(counts, B.hist, sizeof(long long) * S.hist_n, st, e);
    copy_out(wcounts, B.whist, sizeof(double) * S.hist_n, st, e);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
    unsigned long long hc[4] = {0, 0, 0, 0};
    int hblk = 0;
    if (ev.on) {
        PC_CUDA(cudaMemcpyAsync(hc, B.ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
        PC_CUDA(cudaMemcpyAsync(&hblk, B.sc + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        PC_CUDA(cudaEventRecord(ev.e[4], st));
    }
    PC_CUDA(cudaStreamSynchronize(st));
    fill_stats(stats, S, J.cell_size, hc, hblk, ev.ms(0, 4), ev.ms(1, 2), ev.ms(2, 3),
               launch_count() - launches0);
    return PC_OK;
}

// ---------------------------------------------------------------------------
// captured count graphs (pc_count_batch with use_graph)
// ---------------------------------------------------------------------------
// A graph owns its buffers: the shared workspace may be reallocated by other
// calls, and a graph must keep the addresses it was captured with.
struct GraphEntry {
    int dev = 0;
    std::vector<const pc_grid *> grids;
    int mode = 0, los = 0;
    std::vector<double> ea, eb;
    pc_opts o;
    bool weighted = false;
    Workspace W;
    CountSetup S;
    DevBufs B;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long *h_hist = nullptr;   // pinned copies written by the graph
    double *h_whist = nullptr;
    unsigned long long *h_ctr = nullptr;
    int *h_blocks = nullptr;
    long long kernels = 0;                  // kernel launches inside the graph
    ~GraphEntry() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFreeHost(h_hist);
        cudaFreeHost(h_whist);
        cudaFreeHost(h_ctr);
        cudaFreeHost(h_blocks);
        for (Buf *b : {&W.hist, &W.whist, &W.counters, &W.scalars, &W.queue, &W.blocks, &W.tmp_cnt,
                       &W.tmp_off, &W.tmp_tot, &W.tasks, &W.stencil, &W.lut, &W.ea, &W.eb, &W.fold})
            if (b->p) cudaFree(b->p);
    }
};

static std::vector<std::unique_ptr<GraphEntry>> &graph_cache() {
    static std::vector<std::unique_ptr<GraphEntry>> c;
    return c;
}

// Drop every cached graph that uses grid g (called when g is freed).
void forget_grid(const pc_grid *g) {
    auto &c = graph_cache();
    for (size_t k = 0; k < c.size();) {
        bool uses = false;
        for (auto *x : c[k]->grids) uses = uses || (x == g);
        if (uses) c.erase(c.begin() + k); else ++k;
    }
}

static bool same_opts(const pc_opts &a, const pc_opts &b) {
    return a.prec == b.prec && a.cell_size == b.cell_size && a.ipt == b.ipt && a.priv == b.priv &&
           a.rescue_capacity == b.rescue_capacity && a.grid_ctas_per_sm == b.grid_ctas_per_sm &&
           a.shard_index == b.shard_index && a.shard_count == b.shard_count;
}

static pc_status run_count_graph(const CountJob &J, const std::vector<const pc_grid *> &grids,
                                 const pc_bins *b, const pc_opts *opt, cudaStream_t st,
                                 long long *counts, double *wcounts, pc_stats *stats) {
    pc_opts o;
    memset(&o, 0, sizeof(o));
    o.priv = -1;
    if (opt) o = *opt;
    const bool weighted = wcounts != nullptr;
    if (!b || !b->edges_a || (b->mode != PC_BIN_S && !b->edges_b))
        return fail(PC_EINVAL, "bins: missing edges");
    std::vector<double> ea(b->edges_a, b->edges_a + std::max(b->n_a, 0) + 1);
    std::vector<double> eb;
    if (b->mode != PC_BIN_S) eb.assign(b->edges_b, b->edges_b + std::max(b->n_b, 0) + 1);
    GraphEntry *G = nullptr;
    for (auto &c : graph_cache())
        if (c->dev == J.device && c->grids == grids && c->mode == b->mode && c->los == b->los &&
            c->ea == ea && c->eb == eb && same_opts(c->o, o) && c->weighted == weighted)
            G = c.get();
    const long long launches0 = launch_count();
    if (!G) {
        std::unique_ptr<GraphEntry> N(new GraphEntry());
        N->dev = J.device;
        N->grids = grids;
        N->mode = b->mode;
        N->los = b->los;
        N->ea = ea;
        N->eb = eb;
        N->o = o;
        N->weighted = weighted;
        pc_status s = setup_count(J, b, &o, weighted, N->S);
        if (s != PC_OK) return s;
        s = ensure_bufs(N->W, N->S, N->B);
        if (s != PC_OK) return s;
        PairParams p;
        int grid = 0;
        size_t smem = 0;
        s = make_params(J, N->S, N->B, p, grid, smem);
        if (s == PC_OK) s = attach_fold(N->W, p, grid);
        if (s != PC_OK) return s;
        N->S.wsum = p.wint ? (p.wcorr ? 3 : 2) : (N->S.weighted ? 1 : 0);
        const size_t hb = N->S.hist_n;
        PC_CUDA(::pc::alloc_host(&N->h_hist, sizeof(unsigned long long) * hb));
        if (weighted) PC_CUDA(::pc::alloc_host(&N->h_whist, sizeof(double) * hb));
        PC_CUDA(::pc::alloc_host(&N->h_ctr, sizeof(unsigned long long) * 4));
        PC_CUDA(::pc::alloc_host(&N->h_blocks, sizeof(int)));
        cudaStream_t cap = nullptr;
        PC_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        s = upload_tables(J, N->S, N->B, cap);
        if (s == PC_OK) {
            cudaError_t e = cudaStreamSynchronize(cap);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) s = cuda_fail(e, "graph capture");
        }
        if (s == PC_OK) {
            const long long k0 = launch_count();
            s = enqueue_count(N->S, N->B, p, grid, smem, cap, nullptr, nullptr, nullptr);
            N->kernels = launch_count() - k0;
            cudaError_t e = cudaSuccess;
            if (s == PC_OK) {
                e = cudaMemcpyAsync(N->h_hist, N->B.hist, sizeof(unsigned long long) * hb,
                                    cudaMemcpyDeviceToHost, cap);
                if (e == cudaSuccess && weighted)
                    e = cudaMemcpyAsync(N->h_whist, N->B.whist, sizeof(double) * hb,
                                        cudaMemcpyDeviceToHost, cap);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(N->h_ctr, N->B.ctr, sizeof(unsigned long long) * 4,
                                        cudaMemcpyDeviceToHost, cap);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(N->h_blocks, N->B.sc + 1, sizeof(int),
                                        cudaMemcpyDeviceToHost, cap);
            }
            cudaError_t e2 = cudaStreamEndCapture(cap, &N->graph);
            if (s == PC_OK && e != cudaSuccess) s = cuda_fail(e, "graph capture copy");
            if (s == PC_OK && e2 != cudaSuccess) s = cuda_fail(e2, "graph capture end");
            if (s == PC_OK) {
                e = cudaGraphInstantiate(&N->exec, N->graph, 0);
                if (e != cudaSuccess) s = cuda_fail(e, "graph instantiate");
            }
        }
        cudaStreamDestroy(cap);
        if (s != PC_OK) return s;
        graph_cache().push_back(std::move(N));
        G = graph_cache().back().get();
    }
    Events ev(stats != nullptr);
    if (ev.on) PC_CUDA(cudaEventRecord(ev.e[0], st));
    PC_CUDA(cudaGraphLaunch(G->exec, st));
    note_launch((int)G->kernels);   // a replay launches the captured kernels again
    if (ev.on) PC_CUDA(cudaEventRecord(ev.e[4], st));
    PC_CUDA(cudaStreamSynchronize(st));
    const size_t hb = G->S.hist_n;
    cudaError_t e = cudaSuccess;
    if (counts) {
        if (is_device_ptr(counts))
            e = cudaMemcpy(counts, G->h_hist, sizeof(long long) * hb, cudaMemcpyHostToDevice);
        else
            memcpy(counts, G->h_hist, sizeof(long long) * hb);
    }
    if (wcounts && e == cudaSuccess) {
        if (is_device_ptr(wcounts))
            e = cudaMemcpy(wcounts, G->h_whist, sizeof(double) * hb, cudaMemcpyHostToDevice);
        else
            memcpy(wcounts, G->h_whist, sizeof(double) * hb);
    }
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
    unsigned long long hc[4] = {G->h_ctr[0], G->h_ctr[1], G->h_ctr[2], G->h_ctr[3]};
    fill_stats(stats, G->S, J.cell_size, hc, *G->h_blocks, ev.ms(0, 4), 0.f, 0.f,
               launch_count() - launches0);
    return PC_OK;
}

static TaskDev task_of(const pc_grid *gi, const pc_grid *gj, int hist, int is_auto) {
    TaskDev t;
    t.gi = GridDev{gi->rel, gi->cx, gi->xw, gi->cell_start, gi->n, gi->wlo};
    t.gj = GridDev{gj->rel, gj->cx, gj->xw, gj->cell_start, gj->n, gj->wlo};
    t.hist = hist;
    t.is_auto = is_auto;
    // one unit of the integer weight products: 2^(emax_i + emax_j - 300)
    // (w = M 2^(e - 150) with the 24-bit significand M and biased exponent e);
    // the packed significands' product is shifted down by both ranges
    t.wscale = (gi->wint && gj->wint) ? ldexp(1.0, gi->wemax + gj->wemax - 300) : 0.0;
    return t;
}

static bool same_geometry(const pc_grid *a, const pc_grid *b) {
    if (a->g.periodic != b->g.periodic) return false;
    for (int k = 0; k < 3; ++k) {
        if (a->g.ng[k] != b->g.ng[k] || a->g.c[k] != b->g.c[k] || a->g.lo[k] != b->g.lo[k] ||
            a->g.L[k] != b->g.L[k])
            return false;
    }
    return a->device == b->device;
}

}  // namespace pc

using namespace pc;

extern "C" pc_status pc_count_auto(const pc_grid *g, const pc_bins *b, const pc_opts *o,
                                   void *stream, long long *counts, double *wcounts,
                                   pc_stats *st) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!g) return fail(PC_EINVAL, "pc_count_auto: grid is NULL");
    if (!counts && !wcounts) return fail(PC_EINVAL, "pc_count_auto: no output buffer");
    if (wcounts && !g->weighted) return fail(PC_EINVAL, "pc_count_auto: grid has no weights");
    CountJob J;
    J.tasks.push_back(task_of(g, g, 0, 1));
    J.nhist = 1;
    J.is_auto = true;
    job_set_grid(J, g);
    job_add_bounds(J, g, true);
    job_add_wint(J, g, g);
    return run_count(J, b, o, (cudaStream_t)stream, counts, wcounts, st);
}

extern "C" pc_status pc_count_cross(const pc_grid *g1, const pc_grid *g2, const pc_bins *b,
                                    const pc_opts *o, void *stream, long long *counts,
                                    double *wcounts, pc_stats *st) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!g1 || !g2) return fail(PC_EINVAL, "pc_count_cross: grid is NULL");
    if (!counts && !wcounts) return fail(PC_EINVAL, "pc_count_cross: no output buffer");
    if (!same_geometry(g1, g2))
        return fail(PC_EINVAL, "pc_count_cross: grids differ in box, bounds or cell size");
    if (wcounts && !(g1->weighted && g2->weighted))
        return fail(PC_EINVAL, "pc_count_cross: both grids need weights for weighted counts");
    CountJob J;
    J.tasks.push_back(task_of(g1, g2, 0, 0));
    J.nhist = 1;
    J.is_auto = false;
    job_set_grid(J, g1);
    job_add_bounds(J, g1, true);
    job_add_bounds(J, g2, false);
    job_add_wint(J, g1, g2);
    return run_count(J, b, o, (cudaStream_t)stream, counts, wcounts, st);
}

extern "C" pc_status pc_count_batch(const pc_grid *const *gs, int m, const pc_bins *b,
                                    const pc_opts *o, void *stream, long long *counts,
                                    double *wcounts, pc_stats *st) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!gs || m <= 0) return fail(PC_EINVAL, "pc_count_batch: no grids");
    if (m >= (1 << 26)) return fail(PC_EOVERFLOW, "pc_count_batch: too many grids");
    if (!counts && !wcounts) return fail(PC_EINVAL, "pc_count_batch: no output buffer");
    CountJob J;
    for (int k = 0; k < m; ++k) {
        if (!gs[k]) return fail(PC_EINVAL, "pc_count_batch: grid is NULL");
        if (!same_geometry(gs[0], gs[k]))
            return fail(PC_EINVAL, "pc_count_batch: grids differ in box or cell size");
        if (wcounts && !gs[k]->weighted) return fail(PC_EINVAL, "pc_count_batch: grid has no weights");
        J.tasks.push_back(task_of(gs[k], gs[k], k, 1));
        job_add_bounds(J, gs[k], k == 0);
        job_add_wint(J, gs[k], gs[k]);
    }
    J.nhist = m;
    J.is_auto = true;
    job_set_grid(J, gs[0]);
    if (o && o->use_graph) {
        std::vector<const pc_grid *> grids(gs, gs + m);
        return run_count_graph(J, grids, b, o, (cudaStream_t)stream, counts, wcounts, st);
    }
    return run_count(J, b, o, (cudaStream_t)stream, counts, wcounts, st);
}

// ---------------------------------------------------------------------------
// k-d tree counts (Alg. 3): the traversal lists the block pairs, then the
// same pair and rescue kernels as the grid path run over them
// ---------------------------------------------------------------------------
static bool same_tree_geometry(const pc_tree *a, const pc_tree *b) {
    if (a->g.periodic != b->g.periodic || a->device != b->device) return false;
    for (int k = 0; k < 3; ++k)
        if (a->g.L[k] != b->g.L[k]) return false;
    return true;
}

static double tree_rmin(const pc_tree *t) {
    if (t->g.periodic || !(t->r2min > 0.0)) return 0.0;
    return sqrt(t->r2min) * (1.0 - 1e-12);
}

extern "C" pc_status pc_count_tree(const pc_tree *t1, const pc_tree *t2, const pc_bins *b,
                                   const pc_opts *opt, void *stream, long long *counts,
                                   double *wcounts, pc_stats *stats) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!t1) return fail(PC_EINVAL, "pc_count_tree: tree is NULL");
    if (!counts && !wcounts) return fail(PC_EINVAL, "pc_count_tree: no output buffer");
    const bool is_auto = (t2 == nullptr);
    const pc_tree *tj = is_auto ? t1 : t2;
    if (!same_tree_geometry(t1, tj))
        return fail(PC_EINVAL, "pc_count_tree: trees differ in box or device");
    if (wcounts && !(t1->weighted && tj->weighted))
        return fail(PC_EINVAL, "pc_count_tree: weighted counts need weights on every tree");
    cudaStream_t st = (cudaStream_t)stream;

    CountJob J;
    TaskDev T;
    T.gi = GridDev{t1->rel, nullptr, t1->xw, nullptr, t1->n, t1->wlo};
    T.gj = GridDev{tj->rel, nullptr, tj->xw, nullptr, tj->n, tj->wlo};
    T.hist = 0;
    T.is_auto = is_auto ? 1 : 0;
    T.wscale = (t1->wint && tj->wint) ? ldexp(1.0, t1->wemax + tj->wemax - 300) : 0.0;
    J.tasks.push_back(T);
    J.nhist = 1;
    J.is_auto = is_auto;
    J.tree = true;
    // the error bands take the largest block extent where the grid takes
    // the cell side (point offsets from their block centre are at most half
    // of it)
    J.geom = t1->g;
    const double cb = std::max(t1->bext, tj->bext);
    for (int a = 0; a < 3; ++a) {
        J.geom.c[a] = std::max(cb, 1e-300);
        J.geom.c32[a] = (float)J.geom.c[a];
        J.lo[a] = std::min(t1->pts_lo[a], tj->pts_lo[a]);
        J.hi[a] = std::max(t1->pts_hi[a], tj->pts_hi[a]);
        J.plo[a] = J.lo[a];
        J.phi[a] = J.hi[a];
    }
    J.rmin = std::min(tree_rmin(t1), tree_rmin(tj));
    J.device = t1->device;
    J.cell_size = cb;
    if (!t1->wint || !tj->wint ||
        (t1->wemax - t1->wemin) + (tj->wemax - tj->wemin) > WINT_MAX_SPAN)
        J.wint_ok = false;
    if (t1->wcorr || tj->wcorr) J.wcorr = true;

    pc_opts o;
    memset(&o, 0, sizeof(o));
    o.priv = -1;
    if (opt) o = *opt;
    o.ipt = (o.ipt == 4) ? 4 : 2;
    J.ncell = (1 << t1->blevel) * tree_chunks(t1, o.ipt);   // i-blocks (buffer sizes)
    CountSetup S;
    pc_status s = setup_count(J, b, &o, wcounts != nullptr, S);
    if (s != PC_OK) return s;
    if (S.prec != PC_PREC_F32_RESCUE)
        return fail(PC_EUNSUPPORTED,
                    "pc_count_tree: runs the FP32 + rescue kernel only (the plain FP64 path, "
                    "asked for or forced by a midpoint line of sight close to the observer, "
                    "is a grid-path option)");
    DevBufs B;
    s = ensure_bufs(workspace(S.dev), S, B);
    if (s != PC_OK) return s;
    PairParams p;
    int grid = 0;
    size_t smem = 0;
    s = make_params(J, S, B, p, grid, smem);
    if (s == PC_OK) s = attach_fold(workspace(S.dev), p, grid);
    if (s != PC_OK) return s;
    S.wsum = p.wint ? (p.wcorr ? 3 : 2) : (S.weighted ? 1 : 0);
    Events ev(stats != nullptr);
    const long long launches0 = launch_count();
    if (ev.on) PC_CUDA(cudaEventRecord(ev.e[0], st));
    // node pairs closer than the candidate cut, farther than the smallest
    // s edge (the box bounds are exact up to rounding: relative margins)
    const double r2hi = (double)S.P.r2cut * (1.0 + 1e-9);
    const double r2lo = (S.P.mode != PC_BIN_SIGPI) ? S.P.Ea[0] * (1.0 - 1e-9) : 0.0;
    TreeLists TL;
    s = tree_traverse(t1, tj, is_auto, r2hi, r2lo, st, TL);
    if (s != PC_OK) return s;
    p.tseg = TL.seg;
    p.tseg_off = TL.seg_off;
    p.tblk_j = tj->brng;
    p.tcen_i = t1->bcen;
    p.tcen_j = tj->bcen;
    s = upload_tables(J, S, B, st);
    if (s != PC_OK) return s;
    s = enqueue_count(S, B, p, grid, smem, st, ev.e[1], ev.e[2], ev.e[3],
                      [&]() {
                          return tree_blocks(t1, S.ipt, p.shard_index, p.shard_count, B.blocks,
                                             B.sc + 1, st);
                      });
    if (s != PC_OK) return s;
    cudaError_t e = cudaSuccess;
    copy_out(counts, B.hist, sizeof(long long) * S.hist_n, st, e);
    copy_out(wcounts, B.whist, sizeof(double) * S.hist_n, st, e);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
    unsigned long long hc[4] = {0, 0, 0, 0};
    int hblk = 0;
    if (ev.on) {
        PC_CUDA(cudaMemcpyAsync(hc, B.ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
        PC_CUDA(cudaMemcpyAsync(&hblk, B.sc + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        PC_CUDA(cudaEventRecord(ev.e[4], st));
    }
    PC_CUDA(cudaStreamSynchronize(st));
    fill_stats(stats, S, J.cell_size, hc, hblk, ev.ms(0, 4), ev.ms(1, 2), ev.ms(2, 3),
               launch_count() - launches0);
    if (stats) {
        stats->tree_pairs = TL.npairs;
        stats->ms_traverse = ev.ms(0, 1);
    }
    return PC_OK;
}

// Auto counts of m trees in one pair-kernel launch (the tree path's batch):
// each tree is traversed on its own and its lists appended to the batch's.
extern "C" pc_status pc_count_tree_batch(const pc_tree *const *ts, int m, const pc_bins *b,
                                         const pc_opts *opt, void *stream, long long *counts,
                                         double *wcounts, pc_stats *stats) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!ts || m <= 0) return fail(PC_EINVAL, "pc_count_tree_batch: no trees");
    if (m >= (1 << 26)) return fail(PC_EOVERFLOW, "pc_count_tree_batch: too many trees");
    if (!counts && !wcounts) return fail(PC_EINVAL, "pc_count_tree_batch: no output buffer");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<const pc_tree *> trees(ts, ts + m);
    CountJob J;
    double cb = 0.0;
    J.wint_ok = true;
    long long nlist = 0;
    pc_opts o;
    memset(&o, 0, sizeof(o));
    o.priv = -1;
    if (opt) o = *opt;
    o.ipt = (o.ipt == 4) ? 4 : 2;
    for (int k = 0; k < m; ++k) {
        const pc_tree *t = trees[k];
        if (!t) return fail(PC_EINVAL, "pc_count_tree_batch: tree is NULL");
        if (!same_tree_geometry(trees[0], t))
            return fail(PC_EINVAL, "pc_count_tree_batch: trees differ in box or device");
        if (wcounts && !t->weighted)
            return fail(PC_EINVAL, "pc_count_tree_batch: weighted counts need weights on every tree");
        TaskDev T;
        T.gi = GridDev{t->rel, nullptr, t->xw, nullptr, t->n, t->wlo};
        T.gj = T.gi;
        T.hist = k;
        T.is_auto = 1;
        T.wscale = t->wint ? ldexp(1.0, 2 * t->wemax - 300) : 0.0;
        J.tasks.push_back(T);
        cb = std::max(cb, t->bext);
        for (int a = 0; a < 3; ++a) {
            J.lo[a] = k ? std::min(J.lo[a], t->pts_lo[a]) : t->pts_lo[a];
            J.hi[a] = k ? std::max(J.hi[a], t->pts_hi[a]) : t->pts_hi[a];
        }
        J.rmin = k ? std::min(J.rmin, tree_rmin(t)) : tree_rmin(t);
        if (!t->wint || 2 * (t->wemax - t->wemin) > WINT_MAX_SPAN) J.wint_ok = false;
        if (t->wcorr) J.wcorr = true;
        nlist += (long long)(1 << t->blevel) * tree_chunks(t, o.ipt);
    }
    if (nlist >= (1LL << 31)) return fail(PC_EOVERFLOW, "pc_count_tree_batch: too many blocks");
    J.nhist = m;
    J.is_auto = true;
    J.tree = true;
    J.geom = trees[0]->g;
    for (int a = 0; a < 3; ++a) {
        J.geom.c[a] = std::max(cb, 1e-300);
        J.geom.c32[a] = (float)J.geom.c[a];
        J.plo[a] = J.lo[a];
        J.phi[a] = J.hi[a];
    }
    J.device = trees[0]->device;
    // buffers are sized per task x cells: ntasks * ncell covers the blocks
    J.ncell = (int)((nlist + m - 1) / m);
    J.cell_size = cb;
    CountSetup S;
    pc_status s = setup_count(J, b, &o, wcounts != nullptr, S);
    if (s != PC_OK) return s;
    if (S.prec != PC_PREC_F32_RESCUE)
        return fail(PC_EUNSUPPORTED,
                    "pc_count_tree_batch: runs the FP32 + rescue kernel only (see pc_count_tree)");
    DevBufs B;
    s = ensure_bufs(workspace(S.dev), S, B);
    if (s != PC_OK) return s;
    PairParams p;
    int grid = 0;
    size_t smem = 0;
    s = make_params(J, S, B, p, grid, smem);
    if (s == PC_OK) s = attach_fold(workspace(S.dev), p, grid);
    if (s != PC_OK) return s;
    S.wsum = p.wint ? (p.wcorr ? 3 : 2) : (S.weighted ? 1 : 0);
    Events ev(stats != nullptr);
    const long long launches0 = launch_count();
    if (ev.on) PC_CUDA(cudaEventRecord(ev.e[0], st));
    static std::map<int, TreeBatch> batches;   // per device, reused (calls are serialised)
    TreeBatch &TB = batches[S.dev];
    const double r2hi = (double)S.P.r2cut * (1.0 + 1e-9);
    const double r2lo = (S.P.mode != PC_BIN_SIGPI) ? S.P.Ea[0] * (1.0 - 1e-9) : 0.0;
    s = tree_batch_lists(trees, S.ipt, r2hi, r2lo, st, TB);
    if (s != PC_OK) return s;
    p.tseg = (const int2 *)TB.seg.p;
    p.tseg_off = (const int *)TB.off.p;
    p.tblk_j = (const int2 *)TB.rng.p;
    p.tcen_i = (const double *)TB.cen.p;
    p.tcen_j = (const double *)TB.cen.p;
    s = upload_tables(J, S, B, st);
    if (s != PC_OK) return s;
    s = enqueue_count(S, B, p, grid, smem, st, ev.e[1], ev.e[2], ev.e[3], [&]() {
        return tree_blocks_batch(trees, TB, S.ipt, p.shard_index, p.shard_count, B.blocks,
                                 B.sc + 1, st);
    });
    if (s != PC_OK) return s;
    cudaError_t e = cudaSuccess;
    copy_out(counts, B.hist, sizeof(long long) * S.hist_n, st, e);
    copy_out(wcounts, B.whist, sizeof(double) * S.hist_n, st, e);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
    unsigned long long hc[4] = {0, 0, 0, 0};
    int hblk = 0;
    if (ev.on) {
        PC_CUDA(cudaMemcpyAsync(hc, B.ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
        PC_CUDA(cudaMemcpyAsync(&hblk, B.sc + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        PC_CUDA(cudaEventRecord(ev.e[4], st));
    }
    PC_CUDA(cudaStreamSynchronize(st));
    fill_stats(stats, S, J.cell_size, hc, hblk, ev.ms(0, 4), ev.ms(1, 2), ev.ms(2, 3),
               launch_count() - launches0);
    if (stats) {
        stats->tree_pairs = TB.npairs;
        stats->ms_traverse = ev.ms(0, 1);
    }
    return PC_OK;
}

// Host-only view of the stencil the grid path enumerates (no device work).
extern "C" pc_status pc_stencil(const double cell[3], double r_max, int half, int max_rows,
                                int *rows, int *n_rows) {
    if (!cell || !n_rows || max_rows < 0 || (max_rows > 0 && !rows))
        return fail(PC_EINVAL, "pc_stencil: bad arguments");
    if (!(r_max > 0.0) || !std::isfinite(r_max))
        return fail(PC_EINVAL, "pc_stencil: r_max must be positive and finite");
    Geom g;
    memset(&g, 0, sizeof(g));
    for (int a = 0; a < 3; ++a) {
        if (!(cell[a] > 0.0) || !std::isfinite(cell[a]))
            return fail(PC_EINVAL, "pc_stencil: cell sides must be positive and finite");
        if (r_max / cell[a] > 4096.0) return fail(PC_EOVERFLOW, "pc_stencil: too many cells per axis");
        g.c[a] = cell[a];
        g.ng[a] = 1;
    }
    std::vector<int4> st;
    int kmax[3];
    build_stencil(g, r_max, half != 0, st, kmax);
    *n_rows = (int)st.size();
    if ((int)st.size() > max_rows) return fail(PC_EOVERFLOW, "pc_stencil: max_rows too small");
    for (size_t k = 0; k < st.size(); ++k) {
        rows[4 * k] = st[k].x;
        rows[4 * k + 1] = st[k].y;
        rows[4 * k + 2] = st[k].z;
        rows[4 * k + 3] = st[k].w;
    }
    return PC_OK;
}

// Host-only view of the FP32 path's error bands and bin decisions for a
// count (no device work): make_plan on a geometry built from the arguments.
extern "C" pc_status pc_fp32_bands(const pc_bins *b, const double cell[3], const double lo[3],
                                   const double hi[3], const double L[3], int periodic,
                                   double rmin, double out[19]) {
    if (!b || !cell || !lo || !hi || !out || (periodic && !L))
        return fail(PC_EINVAL, "pc_fp32_bands: bad arguments");
    Geom g;
    memset(&g, 0, sizeof(g));
    g.periodic = periodic ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        if (!(cell[a] > 0.0) || !std::isfinite(cell[a]) || !std::isfinite(lo[a]) ||
            !std::isfinite(hi[a]) || hi[a] < lo[a])
            return fail(PC_EINVAL, "pc_fp32_bands: bad cell sides or bounds");
        if (periodic && (!(L[a] > 0.0) || !std::isfinite(L[a])))
            return fail(PC_EINVAL, "pc_fp32_bands: periodic box needs L > 0");
        g.c[a] = cell[a];
        g.c32[a] = (float)cell[a];
        g.ng[a] = 1;
        g.lo[a] = lo[a];
        g.L[a] = periodic ? L[a] : 0.0;
        g.hL[a] = 0.5 * g.L[a];
    }
    Plan P;
    pc_status s = make_plan(b, g, lo, hi, rmin, false, P, false);
    if (s != PC_OK) return s;
    out[0] = P.eps_a;
    out[1] = P.eps_b;
    out[2] = P.mu_A;
    out[3] = P.mu_B;
    out[4] = P.rcut;
    out[5] = P.fp32_ok;
    out[6] = P.lin;
    out[7] = P.r2cut;
    // floor-based bins, as the kernel receives them
    out[8] = P.lin_invA;
    out[9] = P.lin_norange ? P.lin_offA : P.lin_offA1;
    out[10] = P.lin_thrA;
    out[11] = P.lin_nB;
    out[12] = P.lin_mA;
    out[13] = P.lin_cB;
    out[14] = P.lin_norange;
    out[15] = P.lin_log;
    out[16] = P.lin_invB2;
    out[17] = P.lin_thrB;
    out[18] = P.lin_mS;
    return PC_OK;
}

// Host-only copy of the lookup tables a count's FP32 path would stage (the
// same plan as pc_fp32_bands).
extern "C" pc_status pc_fp32_tables(const pc_bins *b, const double cell[3], const double lo[3],
                                    const double hi[3], const double L[3], int periodic,
                                    double rmin, float *lut, int max_entries, int *n_entries,
                                    double desc[7]) {
    if (!b || !cell || !lo || !hi || !n_entries || !desc || (periodic && !L) ||
        max_entries < 0 || (max_entries > 0 && !lut))
        return fail(PC_EINVAL, "pc_fp32_tables: bad arguments");
    Geom g;
    memset(&g, 0, sizeof(g));
    g.periodic = periodic ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        if (!(cell[a] > 0.0) || !std::isfinite(cell[a]) || !std::isfinite(lo[a]) ||
            !std::isfinite(hi[a]) || hi[a] < lo[a])
            return fail(PC_EINVAL, "pc_fp32_tables: bad cell sides or bounds");
        if (periodic && (!(L[a] > 0.0) || !std::isfinite(L[a])))
            return fail(PC_EINVAL, "pc_fp32_tables: periodic box needs L > 0");
        g.c[a] = cell[a];
        g.c32[a] = (float)cell[a];
        g.ng[a] = 1;
        g.lo[a] = lo[a];
        g.L[a] = periodic ? L[a] : 0.0;
        g.hL[a] = 0.5 * g.L[a];
    }
    Plan P;
    pc_status s = make_plan(b, g, lo, hi, rmin, false, P, false);
    if (s != PC_OK) return s;
    *n_entries = (int)P.lut.size();
    desc[0] = P.la.off;
    desc[1] = P.la.T;
    desc[2] = P.la.inv_w;
    desc[3] = P.lb.off;
    desc[4] = P.lb.T;
    desc[5] = P.lb.inv_w;
    desc[6] = P.mu_W;
    if ((int)P.lut.size() > max_entries)
        return fail(PC_EOVERFLOW, "pc_fp32_tables: max_entries too small");
    for (size_t k = 0; k < P.lut.size(); ++k) {
        lut[2 * k] = P.lut[k].x;
        lut[2 * k + 1] = P.lut[k].y;
    }
    return PC_OK;
}

// Cost model of Appendix B.1 (cost = a N_pair + b N_node), specialised to the
// GPU kernel: candidate pairs are charged per thread lane (a block occupies
// NT * 2 lanes however many points its cell holds), and every (block,
// stencil row) visit costs a fixed amount of segment building.
extern "C" double pc_suggest_cell_size(long long n, double volume, double r_max, int mode) {
    (void)mode;
    if (!(r_max > 0.0)) return 1.0;
    if (n <= 1 || !(volume > 0.0)) return r_max;
    const double rho = (double)n / volume;
    const double bi = 2.0 * NT;
    const double a = 1.0, brow = 350.0;   // relative costs (lane-pair, block-row)
    double best = r_max, best_cost = INFINITY;
    for (int k = 2; k <= 64; ++k) {
        double c = r_max * 4.0 / k;   // c from 2 R down to R / 16
        double nc = rho * c * c * c;
        if (nc < 4.0 && k > 2) continue;
        double cells = volume / (c * c * c);
        double blocks_per_cell = std::max(1.0, ceil(nc / bi));
        // stencil cells (half shell) by direct count
        double kk = ceil(r_max / c) + 1;
        double ncand_cells = 0, nrows = 0;
        for (int dz = -(int)kk; dz <= (int)kk; ++dz)
            for (int dy = -(int)kk; dy <= (int)kk; ++dy) {
                double my = std::max(std::abs(dy) - 1, 0) * c, mz = std::max(std::abs(dz) - 1, 0) * c;
                double m2 = my * my + mz * mz;
                if (m2 >= r_max * r_max) continue;
                int rx = 0;
                while (true) {
                    double mx = rx * c;
                    if (mx * mx + m2 < r_max * r_max) ++rx; else break;
                }
                ncand_cells += 2 * rx + 1;
                nrows += 1;
            }
        ncand_cells *= 0.5;
        nrows *= 0.5;
        double lanes = cells * blocks_per_cell * bi;
        double cost = a * lanes * ncand_cells * nc + brow * cells * blocks_per_cell * nrows;
        if (cost < best_cost) {
            best_cost = cost;
            best = c;
        }
    }
    return best;
}

extern "C" const char *pc_strerror(pc_status s) {
    switch (s) {
        case PC_OK: return "success";
        case PC_EINVAL: return "invalid argument";
        case PC_ENOMEM: return "out of memory";
        case PC_ECUDA: return "CUDA error";
        case PC_EOVERFLOW: return "size overflow";
        case PC_ETIMEOUT: return "device wait timed out";
        case PC_EUNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

extern "C" const char *pc_last_error(void) { return g_last_error.c_str(); }

extern "C" long long pc_launch_count(void) { return launch_count(); }

extern "C" long long pc_alloc_count(void) { return alloc_count(); }

extern "C" const char *pc_version(void) { return "paircount-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// Auto counts without device allocation.
//
// For callers that must not allocate device memory at count time: code whose
// device memory is owned by another allocator (a framework's caching
// allocator that holds the whole device), loops that must never hit the
// implicit device synchronisation a cudaMalloc/cudaFree can trigger, and
// processes running at their memory limit.  Every temporary of the count
// lives in one file-scope device array of fixed size instead.
// ---------------------------------------------------------------------------
namespace pc {

// Limits of the fixed scratch array (the call rejects anything larger).
constexpr int NA_MAX_BINS = 16384;        // histogram bins
constexpr int NA_MAX_EDGES = 16385;       // edges per axis
constexpr int NA_MAX_CELLS = 1 << 18;     // cells of the grid
constexpr int NA_MAX_BLOCKS = 1 << 19;    // i-blocks
constexpr int NA_MAX_ROWS = 8192;         // stencil rows
constexpr int NA_MAX_LUT = 2 * (MAX_LUT + 2);
constexpr unsigned long long NA_QUEUE = 1ull << 17;   // rescue slots (overflow is evaluated in-kernel)

struct NaLayout {
    size_t hist, whist, counters, scalars, tasks, stencil, lut, ea, eb, cnt, off, tot, blocks, queue,
        total;
};

constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }

constexpr NaLayout na_layout() {
    NaLayout L{};
    size_t o = 0;
    L.hist = o;     o = na_align(o + sizeof(unsigned long long) * NA_MAX_BINS);
    L.whist = o;    o = na_align(o + sizeof(double) * NA_MAX_BINS);
    L.counters = o; o = na_align(o + sizeof(unsigned long long) * 4);
    L.scalars = o;  o = na_align(o + sizeof(int) * 4);
    L.tasks = o;    o = na_align(o + sizeof(TaskDev));
    L.stencil = o;  o = na_align(o + sizeof(int4) * NA_MAX_ROWS);
    L.lut = o;      o = na_align(o + sizeof(float2) * NA_MAX_LUT);
    L.ea = o;       o = na_align(o + sizeof(double) * NA_MAX_EDGES);
    L.eb = o;       o = na_align(o + sizeof(double) * NA_MAX_EDGES);
    L.cnt = o;      o = na_align(o + sizeof(int) * (NA_MAX_CELLS + 1));
    L.off = o;      o = na_align(o + sizeof(int) * (NA_MAX_CELLS + 1));
    L.tot = o;      o = na_align(o + sizeof(int) * (NA_MAX_CELLS / 4096 + 2));
    L.blocks = o;   o = na_align(o + sizeof(Block) * NA_MAX_BLOCKS);
    L.queue = o;    o = na_align(o + sizeof(uint3) * NA_QUEUE);
    L.total = o;
    return L;
}

constexpr NaLayout NA = na_layout();

// The scratch array (12.3 MiB).  Every GPU that loads the library holds
// it until the process exits.
static __device__ __align__(256) unsigned char g_count_scratch[NA.total];

// Device address of the scratch array on device `dev`, looked up once per
// device with that device current (the host-side symbol is only a stand-in
// and must never be handed to a kernel).
static unsigned char *scratch_on(int dev) {
    static std::map<int, unsigned char *> addr;
    auto it = addr.find(dev);
    if (it != addr.end()) return it->second;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_count_scratch);
    if (e != cudaSuccess) {
        cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        return nullptr;
    }
    addr[dev] = (unsigned char *)p;
    return (unsigned char *)p;
}

}  // namespace pc

extern "C" pc_status pc_count_auto_noalloc(const pc_grid *g, const pc_bins *b, const pc_opts *opt,
                                           void *stream, long long *counts, double *wcounts) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!g) return fail(PC_EINVAL, "pc_count_auto_noalloc: grid is NULL");
    if (!counts && !wcounts) return fail(PC_EINVAL, "pc_count_auto_noalloc: no output buffer");
    if (wcounts && !g->weighted) return fail(PC_EINVAL, "pc_count_auto_noalloc: grid has no weights");
    int cur = -1;
    PC_CUDA(cudaGetDevice(&cur));
    if (cur != g->device)
        return fail(PC_EINVAL, "pc_count_auto_noalloc: the grid's device must be current");
    cudaStream_t st = (cudaStream_t)stream;
    pc_opts o;
    memset(&o, 0, sizeof(o));
    o.priv = -1;
    if (opt) o = *opt;

    if (o.shard_count > 1 && (o.shard_index < 0 || o.shard_index >= o.shard_count))
        return fail(PC_EINVAL, "opts: shard_index must lie in [0, shard_count)");
    Plan P;
    pc_status s = make_plan(b, g->g, g->pts_lo, g->pts_hi, grid_rmin(g), true, P);
    if (s != PC_OK) return s;
    int prec = o.prec;
    if (prec == PC_PREC_F32_RESCUE && !P.fp32_ok) prec = PC_PREC_F64;
    int ipt = (o.ipt == 4) ? 4 : 2;
    if (prec == PC_PREC_F64) ipt = 1;
    const int bi = NT * ipt;
    const long long nblk = (long long)g->ncell + g->n / bi + 16;
    if (P.nbins > NA_MAX_BINS || P.na + 1 > NA_MAX_EDGES || P.nb + 1 > NA_MAX_EDGES)
        return fail(PC_EOVERFLOW, "pc_count_auto_noalloc: more than 16384 bins");
    if (g->ncell > NA_MAX_CELLS)
        return fail(PC_EOVERFLOW, "pc_count_auto_noalloc: grid has more than 262144 cells");
    if (nblk > NA_MAX_BLOCKS)
        return fail(PC_EOVERFLOW, "pc_count_auto_noalloc: more than 524288 point blocks");
    if ((int)P.stencil.size() > NA_MAX_ROWS)
        return fail(PC_EOVERFLOW, "pc_count_auto_noalloc: stencil has more than 8192 rows");
    if ((int)P.lut.size() > NA_MAX_LUT)
        return fail(PC_EOVERFLOW, "pc_count_auto_noalloc: lookup tables too large");

    unsigned char *base = scratch_on(cur);
    if (!base) return PC_ECUDA;
    unsigned long long *hist = (unsigned long long *)(base + NA.hist);
    double *whist = (double *)(base + NA.whist);
    unsigned long long *ctr = (unsigned long long *)(base + NA.counters);
    int *sc = (int *)(base + NA.scalars);
    TaskDev *tasks = (TaskDev *)(base + NA.tasks);

    // everything that must start at zero is cleared on every call
    const size_t hist_n = (size_t)P.nbins;
    PC_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * hist_n, st));
    if (wcounts) PC_CUDA(cudaMemsetAsync(whist, 0, sizeof(double) * hist_n, st));
    PC_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * 4, st));
    PC_CUDA(cudaMemsetAsync(sc, 0, sizeof(int) * 4, st));
    TaskDev t = task_of(g, g, 0, 1);
    PC_CUDA(cudaMemcpyAsync(tasks, &t, sizeof(TaskDev), cudaMemcpyHostToDevice, st));
    if (!P.stencil.empty())
        PC_CUDA(cudaMemcpyAsync(base + NA.stencil, P.stencil.data(), sizeof(int4) * P.stencil.size(),
                                cudaMemcpyHostToDevice, st));
    if (!P.lut.empty())
        PC_CUDA(cudaMemcpyAsync(base + NA.lut, P.lut.data(), sizeof(float2) * P.lut.size(),
                                cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaMemcpyAsync(base + NA.ea, P.Ea.data(), sizeof(double) * (P.na + 1),
                            cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaMemcpyAsync(base + NA.eb, P.Eb.data(), sizeof(double) * (P.nb + 1),
                            cudaMemcpyHostToDevice, st));
    PC_CUDA(make_blocks_into(tasks, 1, g->ncell, bi, o.shard_count > 1 ? o.shard_index : 0,
                             o.shard_count > 1 ? o.shard_count : 1, (Block *)(base + NA.blocks), sc + 1,
                             (int *)(base + NA.cnt), (int *)(base + NA.off),
                             (int *)(base + NA.tot), st));

    PairParams p;
    memset(static_cast<void *>(&p), 0, sizeof(p));
    p.groups = 1;
    p.tasks = tasks;
    p.blocks = (const Block *)(base + NA.blocks);
    p.nblocks = sc + 1;
    p.work_counter = sc;
    p.g = g->g;
    p.stencil = (const int4 *)(base + NA.stencil);
    p.nrows = (int)P.stencil.size();
    p.mode = P.mode;
    p.los = P.los;
    p.weighted = wcounts ? 1 : 0;
    p.n_a = P.na;
    p.n_b = P.nb;
    p.nbins = P.nbins;
    p.r2cut = P.r2cut;
    p.lut = (const float2 *)(base + NA.lut);
    p.lut_total = (int)P.lut.size();
    p.la = P.la;
    p.lb = P.lb;
    p.eps_a = P.eps_a;
    p.eps_b = P.eps_b;
    p.mu_A = P.mu_A;
    p.mu_B = P.mu_B;
    p.mu_W = P.mu_W;
    p.Ea = (const double *)(base + NA.ea);
    p.Eb = (const double *)(base + NA.eb);
    p.hist = hist;
    p.whist = wcounts ? whist : nullptr;
    p.queue = (uint3 *)(base + NA.queue);
    p.qcount = ctr + 2;
    p.qcap = (prec == PC_PREC_F32_RESCUE) ? NA_QUEUE : 0;
    p.counters = ctr;
    p.shard_count = o.shard_count > 1 ? o.shard_count : 1;
    p.shard_index = o.shard_count > 1 ? o.shard_index : 0;
    choose_replication(o.priv, P.nbins, wcounts != nullptr, p.priv, p.hist_k);
    p.wint_k = 1;   // binary64 weight sums here (no integer weight planes)
    p.lin = (prec == PC_PREC_F32_RESCUE) ? P.lin : 0;
    p.lin_norange = p.lin ? P.lin_norange : 0;
    p.lin_log = p.lin ? P.lin_log : 0;
    p.lin_mS = P.lin_mS;
    p.lin_invB2 = P.lin_invB2;
    p.lin_thrB = P.lin_thrB;
    set_hist_rows(p, P);
    p.lin_invA = P.lin_invA;
    // the range-tested floor bins take t_s + 1 (exact floors down to t_s = -1)
    p.lin_offA = P.lin_norange ? P.lin_offA : P.lin_offA1;
    p.lin_thrA = P.lin_thrA;
    p.lin_nB = P.lin_nB;
    p.lin_mA = P.lin_mA;
    p.lin_cB = P.lin_cB;

    int sms = 0, smem_optin = 0;
    PC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur));
    PC_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cur));
    const int lut_size = p.lut_total;
    for (;;) {
        p.smem_hist_ok = 1;
        p.lut_total = p.lin ? 0 : lut_size;
        size_t need = (prec == PC_PREC_F64) ? pairs_f64_smem(p) : pairs_f32_smem(p, ipt);
        if (need + 256 <= (size_t)smem_optin) break;
        if (shrink_replication(p)) continue;
        p.smem_hist_ok = 0;
        p.lut_total = lut_size;
        break;
    }
    size_t smem = (prec == PC_PREC_F64) ? pairs_f64_smem(p) : pairs_f32_smem(p, ipt);
    if (smem + 256 > (size_t)smem_optin)
        return fail(PC_EUNSUPPORTED, "bins: tables do not fit in shared memory");
    int per_sm = (prec == PC_PREC_F64) ? pairs_f64_ctas_per_sm(p, smem)
                                       : pairs_f32_ctas_per_sm(p, ipt, smem);
    if (per_sm <= 0) return fail(PC_ECUDA, "pair kernel cannot be resident");
    if (o.grid_ctas_per_sm > 0) per_sm = std::min(per_sm, o.grid_ctas_per_sm);
    cudaError_t e = (prec == PC_PREC_F64) ? launch_pairs_f64(p, sms * per_sm, smem, st)
                                          : launch_pairs_f32(p, ipt, sms * per_sm, smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "pair kernel launch");
    if (p.qcap) {
        e = launch_rescue(p, st);
        if (e != cudaSuccess) return cuda_fail(e, "rescue kernel launch");
    }
    if (counts) {
        cudaMemcpyKind k = is_device_ptr(counts) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        PC_CUDA(cudaMemcpyAsync(counts, hist, sizeof(long long) * hist_n, k, st));
    }
    if (wcounts) {
        cudaMemcpyKind k = is_device_ptr(wcounts) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        PC_CUDA(cudaMemcpyAsync(wcounts, whist, sizeof(double) * hist_n, k, st));
    }
    PC_CUDA(cudaStreamSynchronize(st));
    return PC_OK;
}
