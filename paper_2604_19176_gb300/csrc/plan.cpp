// plan.cpp — host-side plan builder: geometry tables, the FP64 Abel weights,
// circular-mean work units, CTA schedules and tiles, device upload.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <queue>
#include <thread>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.h"
#include "plan.h"

namespace patgpu {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

template <typename F>
void parallel_for(int n, F&& fn)
{
    int nt = (int)std::thread::hardware_concurrency();
    nt = std::max(1, std::min(nt, 32));
    if (n < 2 || nt == 1) {
        for (int i = 0; i < n; ++i) fn(i);
        return;
    }
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    for (int t = 0; t < std::min(nt, n); ++t)
        th.emplace_back([&]() {
            for (int i = next++; i < n; i = next++) fn(i);
        });
    for (auto& x : th) x.join();
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = kTwoPi / 2;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Product-integration weights w_m(tau) = int_0^tau hat_m(rho) rho / sqrt(tau^2 - rho^2) drho
// (dimensionless; hat_m the piecewise-linear hat on the integer nodes).  The
// substitution rho = tau sin(theta) turns each segment integral into the
// smooth integral of hat(tau sin theta) tau sin theta over theta, evaluated
// with Gauss-Legendre quadrature in FP64.
void abel_weights_gl(double tau, int n_r, const std::vector<double>& gx, const std::vector<double>& gw,
                     double* w)
{
    std::fill(w, w + n_r, 0.0);
    for (int s = 0; s + 1 < n_r && (double)s < tau; ++s) {
        const double a = s, b = std::min((double)(s + 1), tau);
        const double ta = std::asin(a / tau), tb = std::asin(std::min(b / tau, 1.0));
        const double half = 0.5 * (tb - ta), mid = 0.5 * (tb + ta);
        double up = 0.0, dn = 0.0;
        for (size_t i = 0; i < gx.size(); ++i) {
            const double rho = tau * std::sin(mid + half * gx[i]);
            const double wr = gw[i] * rho;
            up += wr * (rho - a);
            dn += wr * (a + 1.0 - rho);
        }
        w[s + 1] += half * up;
        w[s] += half * dn;
    }
}

// Abel-plus-midpoint-derivative matrix P (n_t x (n_t + 2)), FP64 -> FP32:
// p(t_k) = (Q(t_k + Delta/2) - Q(t_k - Delta/2)) / Delta with Q the Abel
// integral of the piecewise-linear circular mean; Delta cancels.
std::vector<float> build_abel_matrix_uncached(int n_t);

// Abel matrices are geometry independent (only n_t matters): cache them.
std::vector<float> build_abel_matrix(int n_t)
{
    static std::mutex mu;
    static std::map<int, std::vector<float>> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(n_t);
        if (it != cache.end()) return it->second;
    }
    std::vector<float> P = build_abel_matrix_uncached(n_t);
    std::lock_guard<std::mutex> lk(mu);
    cache[n_t] = P;
    return P;
}

std::vector<float> build_abel_matrix_uncached(int n_t)
{
    const int n_r = n_t + 2;
    std::vector<double> gx, gw;
    gauss_legendre(12, gx, gw);
    std::vector<double> wt((size_t)(n_t + 1) * n_r);
    parallel_for(n_t + 1, [&](int i) { abel_weights_gl(i + 0.5, n_r, gx, gw, &wt[(size_t)i * n_r]); });
    std::vector<float> P((size_t)n_t * n_r);
    for (int k = 1; k <= n_t; ++k)
        for (int m = 0; m < n_r; ++m)
            P[(size_t)(k - 1) * n_r + m] = (float)(wt[(size_t)k * n_r + m] - wt[(size_t)(k - 1) * n_r + m]);
    return P;
}

struct GeomKey {
    int n, n_det, n_t, K, ml, qp, tw, th;
    double a0, span, tmax;
    bool operator<(const GeomKey& o) const
    {
        return std::tie(n, n_det, n_t, K, ml, qp, tw, th, a0, span, tmax) <
               std::tie(o.n, o.n_det, o.n_t, o.K, o.ml, o.qp, o.tw, o.th, o.a0, o.span, o.tmax);
    }
};

struct TileTemplate {
    int x0, x1, y0, y1;              // owned pixels [x0, x1) x [y0, y1)
    std::vector<Unit> units;         // the tile's units, largest first
    double cost = 0.0;
};

struct GeomTemplate {
    std::vector<TileTemplate> tiles;
    std::vector<int32_t> slotcnt;    // n_det x nmb
    int n_slots = 0;
    int nmb = 0;
    int64_t slot_samples = 0;        // lane-samples the circular-mean kernel evaluates
};

constexpr double kUnitOverhead = 24.0; // per-unit fixed cost, in angle iterations
constexpr double kListTailShare = 0.25; // list gather: share of the work in the shared tail queue

// n pixels split into parts of at most w pixels, as equal as possible.
std::vector<int> tile_edges(int n, int w)
{
    const int parts = std::max(1, (n + w - 1) / w);
    std::vector<int> e(parts + 1);
    for (int i = 0; i <= parts; ++i) e[i] = (int)(((int64_t)i * n) / parts);
    return e;
}

// Staged cells of a tile tw x th pixels (cell_pitch(tw) per row, th + 3 rows).
int64_t tile_cells(int tw, int th) { return (int64_t)cell_pitch(tw) * (th + 3); }

// Tile shape (pixel columns tw, rows th) of an n x n image when a tile may
// stage `cells` cells: the split with the fewest tiles along x plus along y
// (the least tile-edge length, where units straddling an edge are evaluated
// on both sides), wider tiles on ties.  want_w / want_h > 0 fix a side.
void choose_tile(int n, int64_t cells, int want_w, int want_h, int& tw, int& th)
{
    int best = 1 << 30;
    tw = th = 0;
    for (int tx = 1; tx <= n; ++tx) {
        const int w = want_w > 0 ? std::min(want_w, n) : (n + tx - 1) / tx;
        if (want_w > 0 && tx > 1) break;
        int h = want_h > 0 ? std::min(want_h, n) : (int)std::min<int64_t>(n, cells / cell_pitch(w) - 3);
        if (h < 1) continue;
        if (want_h == 0 && tile_cells(w, h) > cells) continue;
        const int ntx = (n + w - 1) / w, nty = (n + h - 1) / h;
        if (ntx + nty < best) {
            best = ntx + nty;
            tw = w;
            th = h;
        }
        if (w <= 8) break;
    }
    if (tw == 0) {   // nothing fits the budget: smallest tiles (the caller checks the shared memory)
        tw = want_w > 0 ? std::min(want_w, n) : std::min(n, 8);
        th = want_h > 0 ? std::min(want_h, n) : std::min(n, 8);
    }
}

} // namespace

static_assert(sizeof(InstDev) % 8 == 0, "InstDev layout");
static_assert(sizeof(Unit) == 32, "Unit layout");

pat_status_t build_plan(Plan& P, const pat_geometry_t* geoms, int n_inst, const pat_options_t& opt,
                        cudaStream_t st)
{
    P.n_inst = n_inst;
    P.geoms.assign(geoms, geoms + n_inst);
    P.opt = opt;
    const bool bf16 = opt.image_dtype == PAT_BF16;
    const int ml = opt.m_lanes;
    const int qpiece = opt.q_piece;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PAT_ERR_CUDA;
    P.device = dev;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return PAT_ERR_CUDA;
    P.num_sms = prop.multiProcessorCount;
    P.max_smem_optin = (int)prop.sharedMemPerBlockOptin;

    // ---- offsets ----------------------------------------------------------
    P.f_offsets.assign(n_inst + 1, 0);
    P.g_offsets.assign(n_inst + 1, 0);
    for (int i = 0; i < n_inst; ++i) {
        P.f_offsets[i + 1] = P.f_offsets[i] + (int64_t)geoms[i].n * geoms[i].n;
        P.g_offsets[i + 1] = P.g_offsets[i] + (int64_t)geoms[i].n_det * geoms[i].n_t;
    }

    // ---- distinct n_t (Abel matrices P, then P^T) --------------------------
    std::map<int, int64_t> p_off;
    std::vector<float> pmat;
    for (int i = 0; i < n_inst; ++i) {
        const int nt = geoms[i].n_t;
        if (!p_off.count(nt)) {
            // P (ntp rows, pitch nrp) then P^T (nrp rows, pitch ntp); padding is
            // zero, so the time kernels' 32-row chunks never leave the matrix.
            // Then the same values in 32 x 32 blocks for the fused time stage,
            // where lane l needs output 32 c + l over contraction rows r of the
            // block: float4 q of a block holds rows 4q .. 4q + 3 of the 32
            // outputs in lane order, so a warp reads each float4 as 512
            // contiguous bytes.  Forward blocks (time chunk c, radius block kc),
            // adjoint blocks (radius chunk c, time block kc).
            p_off[nt] = (int64_t)pmat.size();
            const int nr = nt + 2, nrp = (nr + 31) & ~31, ntp = (nt + 31) & ~31;
            std::vector<float> Pm = build_abel_matrix(nt);
            const size_t base = pmat.size(), plane = (size_t)ntp * nrp;
            pmat.resize(base + 4 * plane, 0.0f);
            const size_t nbr = (size_t)nrp / 32, nbt = (size_t)ntp / 32;
            for (int kk = 0; kk < nt; ++kk)
                for (int m = 0; m < nr; ++m) {
                    const float v = Pm[(size_t)kk * nr + m];
                    pmat[base + (size_t)kk * nrp + m] = v;
                    pmat[base + plane + (size_t)m * ntp + kk] = v;
                    pmat[base + 2 * plane + ((kk / 32) * nbr + m / 32) * 1024 + ((m % 32) / 4 * 32 + kk % 32) * 4 +
                         m % 4] = v;
                    pmat[base + 3 * plane + ((m / 32) * nbt + kk / 32) * 1024 + ((kk % 32) / 4 * 32 + m % 32) * 4 +
                         kk % 4] = v;
                }
        }
    }

    // ---- per-geometry templates (tiles, units, slots) ----------------------
    std::map<GeomKey, int> tmpl_index;
    std::vector<GeomTemplate> tmpls;
    std::vector<int> inst_tmpl(n_inst);
    std::vector<float> detU, detV;     // FP32 detector coordinates (host geometry)
    std::vector<float4> det4, rays;
    std::vector<float2> rtrig;
    std::vector<InstDev> inst(n_inst);
    int64_t tile_bytes = 0;
    int tiles_max = 0;
    int K_max = 0;
    for (int i = 0; i < n_inst; ++i) K_max = std::max(K_max, geoms[i].n_angles);
    const int ray_bytes = K_max * (int)sizeof(float4);   // staged beside the tile
    const int64_t cell_budget = std::max<int64_t>(P.band_budget_bytes - ray_bytes, 16 * 1024) / 16;
    const int QL = kWarp / ml;

    for (int i = 0; i < n_inst; ++i) {
        const pat_geometry_t& g = geoms[i];
        const int n = g.n;
        int tw = 0, th = 0;
        choose_tile(n, cell_budget, opt.tile_cols, opt.band_rows, tw, th);
        const std::vector<int> ex = tile_edges(n, tw), ey = tile_edges(n, th);
        const int ntx = (int)ex.size() - 1, nty = (int)ey.size() - 1;
        tiles_max = std::max(tiles_max, ntx * nty);

        InstDev& d = inst[i];
        std::memset(&d, 0, sizeof(d));
        d.n = n;
        d.n_det = g.n_det;
        d.n_t = g.n_t;
        d.n_r = g.n_t + 2;
        d.n_rp = (d.n_r + 31) & ~31;
        d.n_tp = (g.n_t + 31) & ~31;
        d.K = g.n_angles;
        d.c0 = n / 2;
        const double delta = g.t_max * n / (2.0 * g.n_t); // r_m / h = m * delta
        d.delta = (float)delta;
        d.inv_delta = (float)(1.0 / (double)d.delta);
        d.dphi = (float)(kTwoPi / g.n_angles);
        d.inv_dphi = (float)(g.n_angles / kTwoPi);
        d.inv_K = (float)(1.0 / g.n_angles);
        d.nmb = (d.n_r + ml - 1) / ml;
        d.f_off = P.f_offsets[i];
        d.g_off = P.g_offsets[i];
        d.p_off = p_off[g.n_t];
        d.det_off = (int32_t)detU.size();
        for (int j = 0; j < g.n_det; ++j) {
            // split form: Ui = floor(float(U)), and the exact U minus Ui in FP32
            const double th = g.arc_start + (j + 0.5) * g.arc_span / g.n_det;
            const double ue = std::cos(th) * (n / 2.0) - 0.5, ve = std::sin(th) * (n / 2.0) - 0.5;
            const float uf = (float)ue, vf = (float)ve;
            detU.push_back(uf);
            detV.push_back(vf);
            const double ui = std::floor((double)uf), vi = std::floor((double)vf);
            det4.push_back(make_float4((float)ui, (float)vi, (float)(ue - ui), (float)(ve - vi)));
        }
        // M / Mbar row pitch and the adjoint list code q << (jb + mb) | j << mb | m
        {
            auto bits = [](int64_t v) { int b = 0; while ((1ll << b) < v) ++b; return std::max(b, 1); };
            d.code_mbits = bits(d.n_r + 1);      // m_pitch > n_r: column m_pitch - 1 stays zero
            d.m_pitch = 1 << d.code_mbits;
            d.code_jbits = bits(g.n_det);
            P.code_bits_max = std::max(P.code_bits_max, bits(g.n_angles) + d.code_jbits + d.code_mbits);
        }
        // rays: delta (cos, sin)(2 pi q / K) as FP32 hi + lo pairs (2K entries so
        // that angle windows may run past K), and 1/hi for the adjoint's slab test
        d.ray_off = (int64_t)rays.size();
        {
            auto rcp = [](float x) {
                if (std::fabs((double)x) < 1e-30) return 1e30f;
                const double r = 1.0 / (double)x;
                return (float)std::max(-1e30, std::min(1e30, r));
            };
            for (int q = 0; q < 2 * g.n_angles; ++q) {
                const double ph = kTwoPi * (q % g.n_angles) / g.n_angles;
                const double dc = delta * std::cos(ph), ds = delta * std::sin(ph);
                const float ch = (float)dc, sh = (float)ds;
                rays.push_back(make_float4(ch, sh, (float)(dc - (double)ch), (float)(ds - (double)sh)));
                rtrig.push_back(make_float2(rcp(ch), rcp(sh)));
            }
        }

        GeomKey key{n, g.n_det, g.n_t, g.n_angles, ml, qpiece, tw, th, g.arc_start, g.arc_span, g.t_max};
        auto it = tmpl_index.find(key);
        if (it != tmpl_index.end()) {
            inst_tmpl[i] = it->second;
            continue;
        }
        const int ti = (int)tmpls.size();
        tmpl_index[key] = ti;
        inst_tmpl[i] = ti;
        tmpls.emplace_back();
        GeomTemplate& T = tmpls.back();
        T.nmb = d.nmb;
        const int ntiles = ntx * nty;
        T.tiles.resize(ntiles);
        for (int ty = 0; ty < nty; ++ty)
            for (int tx = 0; tx < ntx; ++tx) {
                TileTemplate& tt = T.tiles[ty * ntx + tx];
                tt.x0 = ex[tx];
                tt.x1 = ex[tx + 1];
                tt.y0 = ey[ty];
                tt.y1 = ey[ty + 1];
                tile_bytes = std::max<int64_t>(tile_bytes, 16 * tile_cells(tt.x1 - tt.x0, tt.y1 - tt.y0));
            }
        // Units.  A sample touches tile [x0, x1) x [y0, y1) iff its cell does,
        // i.e. its centred position lies in [x0 - 1 - c0, x1 - c0) x
        // [y0 - 1 - c0, y1 - c0).  For every (detector, radius block, ray) the
        // block's samples lie on one straight segment, so the segment's
        // bounding box (widened by eps, far above the FP32 position error)
        // against those rectangles finds every tile a sample of it can touch.
        // Runs of consecutive rays touching a tile become that tile's units.
        const int c0 = n / 2;
        const double eps = 0.01;
        const int K = g.n_angles;
        std::vector<double> cq(K), sq(K);
        for (int q = 0; q < K; ++q) {
            cq[q] = std::cos(kTwoPi * q / K);
            sq[q] = std::sin(kTwoPi * q / K);
        }
        std::vector<double> rx0(ntx), rx1(ntx), ry0(nty), ry1(nty);
        for (int tx = 0; tx < ntx; ++tx) {
            rx0[tx] = ex[tx] - 1 - c0 - eps;
            rx1[tx] = ex[tx + 1] - c0 + eps;
        }
        for (int ty = 0; ty < nty; ++ty) {
            ry0[ty] = ey[ty] - 1 - c0 - eps;
            ry1[ty] = ey[ty + 1] - c0 + eps;
        }
        std::vector<std::vector<std::vector<Unit>>> per(g.n_det, std::vector<std::vector<Unit>>(ntiles));
        const float* Uj = &detU[d.det_off];
        const float* Vj = &detV[d.det_off];
        parallel_for(g.n_det, [&](int j) {
            std::vector<int> last(ntiles), start(ntiles);
            std::vector<std::vector<std::pair<int, int>>> runs(ntiles);   // [q_begin, q_end)
            for (int mb = 0; mb < d.nmb; ++mb) {
                const int m0 = mb * ml, m1 = std::min(m0 + ml, d.n_r) - 1;
                const double r0 = m0 * delta, r1 = m1 * delta;
                std::fill(last.begin(), last.end(), -2);
                for (auto& r : runs) r.clear();
                for (int q = 0; q < K; ++q) {
                    const double xa = Uj[j] + r0 * cq[q], xb = Uj[j] + r1 * cq[q];
                    const double ya = Vj[j] + r0 * sq[q], yb = Vj[j] + r1 * sq[q];
                    const double bx0 = std::min(xa, xb), bx1 = std::max(xa, xb);
                    const double by0 = std::min(ya, yb), by1 = std::max(ya, yb);
                    if (bx1 < rx0[0] || bx0 > rx1[ntx - 1] || by1 < ry0[0] || by0 > ry1[nty - 1]) continue;
                    for (int ty = 0; ty < nty; ++ty) {
                        if (by1 < ry0[ty] || by0 > ry1[ty]) continue;
                        for (int tx = 0; tx < ntx; ++tx) {
                            if (bx1 < rx0[tx] || bx0 > rx1[tx]) continue;
                            const int t = ty * ntx + tx;
                            if (last[t] != q - 1) {
                                if (last[t] >= 0) runs[t].emplace_back(start[t], last[t] + 1);
                                start[t] = q;
                            }
                            last[t] = q;
                        }
                    }
                }
                for (int t = 0; t < ntiles; ++t) {
                    if (last[t] >= 0) runs[t].emplace_back(start[t], last[t] + 1);
                    auto& rr = runs[t];
                    // a run through q = K - 1 continues at q = 0
                    if (rr.size() >= 2 && rr.front().first == 0 && rr.back().second == K) {
                        rr.back().second = K + rr.front().second;
                        rr.erase(rr.begin());
                    }
                    for (auto& r : rr) {
                        int q0 = r.first, len = r.second - r.first;
                        while (len > 0) {
                            // pieces never wrap past K (the kernel indexes K staged rays)
                            const int qs = q0 % K;
                            const int piece = std::min(std::min(len, qpiece), K - qs);
                            Unit u{};
                            u.j = j;
                            u.m0 = m0;
                            u.q0 = qs;
                            u.nq = piece;
                            per[j][t].push_back(u);
                            q0 += piece;
                            len -= piece;
                        }
                    }
                }
            }
        });
        // slots per (detector, radius block), counted across tiles in order
        T.slotcnt.assign((size_t)g.n_det * d.nmb, 0);
        for (int t = 0; t < ntiles; ++t)
            for (int j = 0; j < g.n_det; ++j)
                for (Unit& u : per[j][t]) {
                    int32_t& cnt = T.slotcnt[(size_t)j * d.nmb + u.m0 / ml];
                    u.slot = cnt++;
                    T.n_slots = std::max(T.n_slots, (int)cnt);
                    T.slot_samples += (int64_t)((u.nq + QL - 1) / QL) * kWarp;
                }
        for (int t = 0; t < ntiles; ++t) {
            auto& tile = T.tiles[t];
            for (int j = 0; j < g.n_det; ++j) tile.units.insert(tile.units.end(), per[j][t].begin(), per[j][t].end());
            for (const Unit& u : tile.units) tile.cost += (double)(u.nq + QL - 1) / QL + kUnitOverhead;
        }
    }

    // ---- CTA schedule for the circular means ------------------------------
    // Tile tasks: (instance, tile).  Each task gets CTAs ("parts") in
    // proportion to its cost (at least one); parts are placed on CTAs by LPT.
    // Within a task, the units are spread over the parts' warps by LPT on
    // their cost (a sample costs the same everywhere), once per template tile
    // and part count, so identical instances share the schedule.
    const int64_t smem_bytes64 = tile_bytes + ray_bytes;
    if (smem_bytes64 > P.max_smem_optin) return PAT_ERR_UNSUPPORTED;
    const int smem_bytes = (int)smem_bytes64;
    P.fwd_smem = smem_bytes;
    const int bps = circmean_blocks_per_sm(ml, bf16, smem_bytes);
    if (bps < 1) return PAT_ERR_UNSUPPORTED;
    const int n_ctas_target = bps * P.num_sms;
    constexpr int kWarpsCta = kCircThreads / kWarp;
    auto unit_cost = [&](const Unit& u) { return (double)((u.nq + QL - 1) / QL) + kUnitOverhead; };
    double total_cost = 0.0;
    for (int i = 0; i < n_inst; ++i)
        for (const auto& tt : tmpls[inst_tmpl[i]].tiles) total_cost += tt.cost;
    // parts per template tile
    std::vector<std::vector<int>> tile_parts(tmpls.size());
    for (size_t t = 0; t < tmpls.size(); ++t) {
        tile_parts[t].resize(tmpls[t].tiles.size(), 0);
        for (size_t k = 0; k < tmpls[t].tiles.size(); ++k) {
            const TileTemplate& tt = tmpls[t].tiles[k];
            if (tt.units.empty()) continue;
            const double share = tt.cost / std::max(total_cost, 1.0) * n_ctas_target;
            const int nunits = (int)tt.units.size();
            tile_parts[t][k] = std::max(1, std::min((int)std::lround(share), std::max(1, nunits / (2 * kWarpsCta))));
        }
    }
    // per (template tile): units grouped by (part, warp); offsets per warp
    std::vector<Unit> units;
    std::vector<int32_t> warp_units;
    std::vector<std::vector<int32_t>> tile_woff(tmpls.size());   // first warp_units index of (tile, part 0)
    for (size_t t = 0; t < tmpls.size(); ++t) {
        tile_woff[t].assign(tmpls[t].tiles.size(), -1);
        for (size_t k = 0; k < tmpls[t].tiles.size(); ++k) {
            const TileTemplate& tt = tmpls[t].tiles[k];
            const int np = tile_parts[t][k];
            if (np == 0) continue;
            const int nw = np * kWarpsCta;
            std::vector<std::vector<Unit>> lists(nw);
            using E = std::pair<double, int>;
            std::priority_queue<E, std::vector<E>, std::greater<E>> pq;
            for (int w = 0; w < nw; ++w) pq.push({0.0, w});
            for (const Unit& u : tt.units) {   // units are sorted largest first
                E e = pq.top();
                pq.pop();
                lists[e.second].push_back(u);
                pq.push({e.first + unit_cost(u), e.second});
            }
            tile_woff[t][k] = (int32_t)warp_units.size();
            for (int w = 0; w < nw; ++w) {
                warp_units.push_back((int32_t)units.size());
                units.insert(units.end(), lists[w].begin(), lists[w].end());
            }
            warp_units.push_back((int32_t)units.size());   // end of the last warp (one slot per tile)
        }
    }
    struct PartC {
        Segment s;
        double cost;
    };
    std::vector<PartC> parts;
    for (int i = 0; i < n_inst; ++i) {
        const int t = inst_tmpl[i];
        const GeomTemplate& T = tmpls[t];
        for (size_t k = 0; k < T.tiles.size(); ++k) {
            const TileTemplate& tt = T.tiles[k];
            const int np = tile_parts[t][k];
            for (int p = 0; p < np; ++p) {
                Segment s{};
                s.inst = i;
                s.x0 = tt.x0;
                s.x1 = tt.x1;
                s.y0 = tt.y0;
                s.y1 = tt.y1;
                s.pitch = cell_pitch(tt.x1 - tt.x0);
                s.warp_off = tile_woff[t][k] + p * kWarpsCta;
                parts.push_back({s, tt.cost / np});
            }
        }
    }
    std::stable_sort(parts.begin(), parts.end(), [](const PartC& a, const PartC& b) { return a.cost > b.cost; });
    const int n_ctas = std::max(1, std::min(n_ctas_target, (int)parts.size()));
    std::vector<std::vector<Segment>> cta_lists(n_ctas);
    {
        using E = std::pair<double, int>;
        std::priority_queue<E, std::vector<E>, std::greater<E>> pq;
        for (int c = 0; c < n_ctas; ++c) pq.push({0.0, c});
        for (const PartC& p : parts) {
            E e = pq.top();
            pq.pop();
            cta_lists[e.second].push_back(p.s);
            pq.push({e.first + p.cost + 8.0 * kUnitOverhead, e.second});
        }
    }
    std::vector<Segment> segs;
    std::vector<int32_t> cta_seg(1, 0);
    for (auto& l : cta_lists) {
        segs.insert(segs.end(), l.begin(), l.end());
        cta_seg.push_back((int32_t)segs.size());
    }
    if (parts.empty()) cta_seg.assign(1, 0);
    std::vector<int2> msum_rows;
    for (int i = 0; i < n_inst; ++i)
        for (int j = 0; j < geoms[i].n_det; ++j) msum_rows.push_back(make_int2(i, j));

    // ---- adjoint cell items -------------------------------------------------
    int64_t patches = 0;
    for (int i = 0; i < n_inst; ++i) {
        const int n = geoms[i].n;
        patches += (int64_t)((n + 1 + kPatchW - 1) / kPatchW) * ((n + 1 + kPatchH - 1) / kPatchH);
    }
    const int cbps = adj_cells_blocks_per_sm();
    if (cbps < 1) return PAT_ERR_UNSUPPORTED;
    const int64_t resident_warps = (int64_t)cbps * P.num_sms * 8;
    // adjoint list mode is chosen here (the sample count used for the budget is
    // the forward's evaluated-sample upper bound).  Instances with the same
    // geometry share one template's lists, so each template counts once.
    int64_t slot_samples_all = 0;
    {
        std::vector<char> seen(tmpls.size(), 0);
        for (int i = 0; i < n_inst; ++i)
            if (!seen[inst_tmpl[i]]) {
                seen[inst_tmpl[i]] = 1;
                slot_samples_all += tmpls[inst_tmpl[i]].slot_samples;
            }
    }
    // packed code lists (4 B per sample; run pairs when a code has a bit to
    // spare) when the code bits and the budget allow (the fastest form
    // measured), else fraction lists (12 B per sample), else enumeration on
    // every call
    const bool codes_fit = P.code_bits_max <= 32, pairs_fit = P.code_bits_max <= 31;
    if (opt.adj_mode == 1 && !codes_fit) return PAT_ERR_UNSUPPORTED;
    if (opt.adj_mode == 4 && !pairs_fit) return PAT_ERR_UNSUPPORTED;
    int list_mode = opt.adj_mode;
    if (list_mode == 0) {
        // (aligned code lists: the budget allows for their null entries)
        const double budget = (double)P.list_budget_bytes;
        list_mode = codes_fit && (double)slot_samples_all * 4.0 * 1.5 <= budget ? (pairs_fit ? 4 : 1)
                    : (double)slot_samples_all * 12.0 <= budget                  ? 3
                                                                                 : 2;
    }
    const bool use_lists = list_mode == 1 || list_mode == 3 || list_mode == 4;
    const bool frac_lists = list_mode == 3;
    const int list_lm = list_mode == 3 ? 1 : list_mode == 4 ? 2 : 0;
    // detectors per aligned block of the code lists (measured best at 8 on
    // the 256^2 - 760^2 workloads; the autotuner tries others)
    const int jblock = use_lists && !frac_lists ? (opt.adj_jblock > 0 ? opt.adj_jblock : 8) : 0;
    int AG = opt.adj_groups;
    if (AG == 0) AG = (int)std::max<int64_t>(1, std::min<int64_t>(16, (2 * resident_warps + patches - 1) / patches));
    // Items with an estimate of their cost (candidate rays per detector, from
    // the patch centre), sorted largest first for the kernel's dynamic queue.
    std::vector<std::pair<double, CellItem>> wit;
    for (int i = 0; i < n_inst; ++i) {
        const InstDev& d = inst[i];
        const int n = geoms[i].n;
        const double R = 0.7111, per_rad = d.K / kTwoPi;
        for (int y0 = -1; y0 <= n - 1; y0 += kPatchH)
            for (int x0 = -1; x0 <= n - 1; x0 += kPatchW) {
                const double px = x0 - d.c0 + 0.5 * kPatchW, py = y0 - d.c0 + 0.5 * kPatchH;
                for (int gg = 0; gg < AG; ++gg) {
                    double cost = 0.0;
                    for (int j = gg; j < d.n_det; j += AG) {
                        const double rc = std::hypot(px - detU[d.det_off + j], py - detV[d.det_off + j]);
                        const double rays = rc <= 1.25 * R ? d.K : 2.0 * std::asin(std::min(1.0, R / rc)) * per_rad + 1;
                        cost += 3.0 + rays;
                    }
                    wit.push_back({cost, CellItem{i, x0, y0, gg}});
                }
            }
    }
    std::stable_sort(wit.begin(), wit.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    // list mode: each cell's list is cut into LG parts (one corner-sum plane
    // each), enough (patch, part) items for about two per resident warp
    int LG = 1;
    if (use_lists) {
        const int lbps = adj_list_blocks_per_sm(list_lm);
        if (lbps < 1) return PAT_ERR_UNSUPPORTED;
        const int64_t lres = (int64_t)lbps * P.num_sms * 8;
        LG = opt.adj_groups > 0 ? opt.adj_groups
                                : (int)std::max<int64_t>(1, std::min<int64_t>(16, (2 * lres + patches - 1) / patches));
    }
    const int ZG = use_lists ? LG : AG;
    std::vector<CellItem> citems;
    citems.reserve(wit.size());
    for (auto& w : wit) citems.push_back(w.second);
    const int cell_blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)cbps * P.num_sms, ((int64_t)citems.size() + 7) / 8));

    // ---- per-instance workspace offsets and slot counts -------------------
    std::vector<int32_t> slotcnt;
    std::map<int, int64_t> tmpl_slot_off;
    int64_t mpart_total = 0, mbar_total = 0, z_total = 0;
    int64_t samples_slots = 0;
    for (int i = 0; i < n_inst; ++i) {
        const int ti = inst_tmpl[i];
        GeomTemplate& T = tmpls[ti];
        if (!tmpl_slot_off.count(ti)) {
            tmpl_slot_off[ti] = (int64_t)slotcnt.size() * 4;
            slotcnt.insert(slotcnt.end(), T.slotcnt.begin(), T.slotcnt.end());
        }
        InstDev& d = inst[i];
        d.slotcnt_off = tmpl_slot_off[ti];
        d.n_slots = T.n_slots;
        d.mpart_off = mpart_total;
        mpart_total += (int64_t)T.n_slots * d.n_det * d.n_r;
        d.mbar_off = mbar_total;
        mbar_total += (int64_t)d.n_det * d.m_pitch;
        d.z_off = z_total;
        z_total += (int64_t)ZG * (d.n + 1) * (d.n + 1);
        samples_slots += T.slot_samples;
    }

    // ---- tiles --------------------------------------------------------------
    std::vector<TimeTile> fwd_tiles, adj_tiles;
    std::vector<ImgTile> itiles;
    int64_t time_macs = 0;
    for (int i = 0; i < n_inst; ++i) {
        const InstDev& d = inst[i];
        for (int j0 = 0; j0 < d.n_det; j0 += kAbelJ) {
            for (int k0 = 0; k0 < d.n_t; k0 += kAbelX) fwd_tiles.push_back({i, j0, k0, 0});
            for (int m0 = 0; m0 < d.n_r; m0 += kAbelX) adj_tiles.push_back({i, j0, m0, 0});
        }
        for (int y0 = 0; y0 < d.n; y0 += 8)
            for (int x0 = 0; x0 < d.n; x0 += 32) itiles.push_back({i, x0, y0, 0});
        // nonzeros of P: rows kk have m <= kk + 2 (kk = k - 1)
        int64_t nnz = 0;
        for (int kk = 0; kk < d.n_t; ++kk) nnz += std::min(kk + 3, d.n_r);
        time_macs += nnz * d.n_det;
    }
    // longest contractions first (the triangle makes late forward tiles and
    // early adjoint tiles heavier)
    auto fwd_len = [&](const TimeTile& t) { return std::min(inst[t.inst].n_r, t.x0 + kAbelX + 2); };
    auto adj_len = [&](const TimeTile& t) { return inst[t.inst].n_t - std::max(0, t.x0 - 2); };
    std::stable_sort(fwd_tiles.begin(), fwd_tiles.end(),
                     [&](const TimeTile& a, const TimeTile& b) { return fwd_len(a) > fwd_len(b); });
    std::stable_sort(adj_tiles.begin(), adj_tiles.end(),
                     [&](const TimeTile& a, const TimeTile& b) { return adj_len(a) > adj_len(b); });
    // fused time stage of the steps: one cluster per kTimeJ detectors (largest
    // n_t first); shared memory per CTA: the group's rows of M and of the
    // residual, the warps' partial sums and the data of its time chunks
    std::vector<TimeGroup> tgroups;
    int time_rows_r = 0, time_rows_t = 0;
    for (int i = 0; i < n_inst; ++i) {
        const InstDev& d = inst[i];
        for (int j0 = 0; j0 < d.n_det; j0 += kTimeJ) tgroups.push_back({i, j0, std::min(kTimeJ, d.n_det - j0), 0});
        time_rows_r = std::max(time_rows_r, d.n_rp);
        time_rows_t = std::max(time_rows_t, d.n_tp);
    }
    std::stable_sort(tgroups.begin(), tgroups.end(),
                     [&](const TimeGroup& a, const TimeGroup& b) { return inst[a.inst].n_t > inst[b.inst].n_t; });
    int time_chunks = 0, time_smem = 0;
    if (opt.time_pair == 0) {
        const int chunks = (time_rows_r / 32 + kTimeCS - 1) / kTimeCS;   // n_rc >= n_tc
        const int64_t bytes = (int64_t)(time_rows_r + time_rows_t) * kTimeJ * 4 +
                              (int64_t)chunks * (kTimeWarps + 2) * kTimeJ * kWarp * 4;
        if (bytes <= P.max_smem_optin && time_pair_clusters((int)bytes) > 0) {
            time_chunks = chunks;
            time_smem = (int)bytes;
        }
    }
    // with fewer tiles than SMs, a cluster of CTAs splits each contraction
    auto cluster_for = [&](size_t tiles) {
        if (opt.abel_split > 0) return (int)opt.abel_split;
        return tiles >= (size_t)P.num_sms ? 1 : tiles * 2 >= (size_t)P.num_sms ? 2 : 4;
    };

    // ---- upload -----------------------------------------------------------
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    auto reserve = [&](size_t bytes) {
        const size_t o = off;
        off = align(off + std::max<size_t>(bytes, 1));
        return o;
    };
    const size_t o_inst = reserve(sizeof(InstDev) * inst.size());
    const size_t o_det = reserve(sizeof(float4) * det4.size());
    const size_t o_rays = reserve(sizeof(float4) * rays.size());
    const size_t o_rtrig = reserve(sizeof(float2) * rtrig.size());
    const size_t o_P = reserve(sizeof(float) * pmat.size());
    const size_t o_slot = reserve(sizeof(int32_t) * slotcnt.size());
    const size_t o_units = reserve(sizeof(Unit) * units.size());
    const size_t o_wunits = reserve(sizeof(int32_t) * warp_units.size());
    const size_t o_msrows = reserve(sizeof(int2) * msum_rows.size());
    const size_t o_segs = reserve(sizeof(Segment) * segs.size());
    const size_t o_ctaseg = reserve(sizeof(int32_t) * cta_seg.size());
    const size_t o_ft = reserve(sizeof(TimeTile) * fwd_tiles.size());
    const size_t o_at = reserve(sizeof(TimeTile) * adj_tiles.size());
    const size_t o_ci = reserve(sizeof(CellItem) * citems.size());
    const size_t o_it = reserve(sizeof(ImgTile) * itiles.size());
    const size_t o_tg = reserve(sizeof(TimeGroup) * tgroups.size());
    const size_t o_status = reserve(64);
    const size_t o_count = reserve(64);
    P.tables_bytes = off;
    if (dev_malloc(&P.d_tables, P.tables_bytes) != cudaSuccess) {
        P.d_tables = nullptr;
        cudaGetLastError();
        return PAT_ERR_OOM;
    }
    std::vector<unsigned char> host(P.tables_bytes, 0);
    auto put = [&](size_t o, const void* src, size_t bytes) {
        if (bytes) std::memcpy(host.data() + o, src, bytes);
    };
    put(o_inst, inst.data(), sizeof(InstDev) * inst.size());
    put(o_det, det4.data(), sizeof(float4) * det4.size());
    put(o_rays, rays.data(), sizeof(float4) * rays.size());
    put(o_rtrig, rtrig.data(), sizeof(float2) * rtrig.size());
    put(o_P, pmat.data(), sizeof(float) * pmat.size());
    put(o_slot, slotcnt.data(), sizeof(int32_t) * slotcnt.size());
    put(o_units, units.data(), sizeof(Unit) * units.size());
    put(o_wunits, warp_units.data(), sizeof(int32_t) * warp_units.size());
    put(o_msrows, msum_rows.data(), sizeof(int2) * msum_rows.size());
    put(o_segs, segs.data(), sizeof(Segment) * segs.size());
    put(o_ctaseg, cta_seg.data(), sizeof(int32_t) * cta_seg.size());
    put(o_ft, fwd_tiles.data(), sizeof(TimeTile) * fwd_tiles.size());
    put(o_at, adj_tiles.data(), sizeof(TimeTile) * adj_tiles.size());
    put(o_ci, citems.data(), sizeof(CellItem) * citems.size());
    put(o_it, itiles.data(), sizeof(ImgTile) * itiles.size());
    put(o_tg, tgroups.data(), sizeof(TimeGroup) * tgroups.size());
    if (cudaMemcpyAsync(P.d_tables, host.data(), P.tables_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return PAT_ERR_CUDA;

    // workspace (floats): forward slots | Mbar | TV partials | (aligned) cell sums (float4)
    // workspace (4-byte words): slots | M | Mbar | TV partials | arrival counters | cell sums (float4)
    const int64_t tv_parts = 3 * (int64_t)itiles.size();
    const int64_t o_msum = mpart_total, o_mbar = o_msum + mbar_total, o_tvp = o_mbar + mbar_total;
    const int64_t o_ctr = ((o_tvp + tv_parts + kQueueStride - 1) / kQueueStride) * kQueueStride;
    const int64_t n_ctr = 2 * (int64_t)kQueueStride;
    const int64_t o_res = ((o_ctr + n_ctr + 63) / 64) * 64;   // data residual of pat_tv_step
    const int64_t z_float_off = ((o_res + P.g_offsets[n_inst] + 63) / 64) * 64;
    P.work_floats = z_float_off + 4 * z_total;
    if (dev_malloc(reinterpret_cast<void**>(&P.d_work), sizeof(float) * std::max<int64_t>(P.work_floats, 1)) !=
        cudaSuccess) {
        P.d_work = nullptr;
        cudaGetLastError();
        return PAT_ERR_OOM;
    }
    // zero everything once: the work-queue counters start (and are left by
    // every call) at 0, and the columns of M and Mbar from n_r on stay zero
    if (cudaMemsetAsync(P.d_work, 0, sizeof(float) * std::max<int64_t>(P.work_floats, 1), st) != cudaSuccess)
        return PAT_ERR_CUDA;

    unsigned char* base = static_cast<unsigned char*>(P.d_tables);
    DevPlan& dp = P.dp;
    std::memset(&dp, 0, sizeof(dp));
    dp.inst = reinterpret_cast<const InstDev*>(base + o_inst);
    dp.det = reinterpret_cast<const float4*>(base + o_det);
    dp.rays = reinterpret_cast<const float4*>(base + o_rays);
    dp.rtrig = reinterpret_cast<const float2*>(base + o_rtrig);
    dp.P = reinterpret_cast<const float*>(base + o_P);
    dp.slotcnt = reinterpret_cast<const uint8_t*>(base + o_slot);
    dp.units = reinterpret_cast<const Unit*>(base + o_units);
    dp.warp_units = reinterpret_cast<const int32_t*>(base + o_wunits);
    dp.msum_rows = reinterpret_cast<const int2*>(base + o_msrows);
    dp.n_msum_rows = (int32_t)msum_rows.size();
    dp.n_r_max = 0;
    for (int i = 0; i < n_inst; ++i) dp.n_r_max = std::max(dp.n_r_max, inst[i].n_r);
    dp.segs = reinterpret_cast<const Segment*>(base + o_segs);
    dp.cta_seg = reinterpret_cast<const int32_t*>(base + o_ctaseg);
    dp.fwd_tiles = reinterpret_cast<const TimeTile*>(base + o_ft);
    dp.adj_tiles = reinterpret_cast<const TimeTile*>(base + o_at);
    dp.cell_items = reinterpret_cast<const CellItem*>(base + o_ci);
    dp.img_tiles = reinterpret_cast<const ImgTile*>(base + o_it);
    dp.time_groups = reinterpret_cast<const TimeGroup*>(base + o_tg);
    dp.n_time_groups = (int32_t)tgroups.size();
    dp.time_chunks = time_chunks;
    dp.time_rows_r = time_rows_r;
    dp.time_rows_t = time_rows_t;
    dp.time_smem_bytes = time_smem;
    dp.mpart = P.d_work;
    dp.msum = P.d_work + o_msum;
    dp.mbar = P.d_work + o_mbar;
    dp.tv_partial = P.d_work + o_tvp;
    dp.work_counters = reinterpret_cast<int32_t*>(P.d_work + o_ctr);
    P.d_resid = P.d_work + o_res;
    P.d_counters = reinterpret_cast<int32_t*>(P.d_work + o_ctr);
    P.counters_bytes = (size_t)n_ctr * 4;
    dp.zbuf = reinterpret_cast<float4*>(P.d_work + z_float_off);
    dp.status = reinterpret_cast<int32_t*>(base + o_status);
    dp.n_inst = n_inst;
    dp.n_fwd_ctas = (int)cta_seg.size() - 1;
    dp.n_fwd_tiles = (int)fwd_tiles.size();
    dp.n_adj_tiles = (int)adj_tiles.size();
    dp.n_cell_items = (int)citems.size();
    dp.n_img_tiles = (int)itiles.size();
    dp.m_lanes = ml;
    dp.adj_groups = AG;
    dp.cell_blocks = cell_blocks;
    dp.fwd_smem_bytes = smem_bytes;
    dp.fwd_rays_off = (int32_t)tile_bytes;
    dp.abel_cluster_fwd = cluster_for(fwd_tiles.size());
    dp.abel_cluster_adj = cluster_for(adj_tiles.size());
    dp.bf16 = bf16 ? 1 : 0;

    // ---- sample count (exact, with the kernels' FP32 arithmetic) ----------
    unsigned long long* d_count = reinterpret_cast<unsigned long long*>(base + o_count);
    if (cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st) != cudaSuccess) return PAT_ERR_CUDA;
    // once per geometry template (identical instances have identical counts)
    unsigned long long count = 0;
    {
        std::vector<int> mult(tmpls.size(), 0), first(tmpls.size(), -1);
        for (int i = 0; i < n_inst; ++i) {
            if (first[inst_tmpl[i]] < 0) first[inst_tmpl[i]] = i;
            ++mult[inst_tmpl[i]];
        }
        for (size_t t = 0; t < tmpls.size(); ++t) {
            const int i = first[t];
            unsigned long long c = 0;
            if (cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st) != cudaSuccess ||
                launch_count_samples(dp, i, inst[i].n_det, d_count, st) != cudaSuccess ||
                cudaMemcpyAsync(&c, d_count, sizeof(c), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return PAT_ERR_CUDA;
            count += c * (unsigned long long)mult[t];
        }
    }

    // ---- adjoint sample lists (list mode) --------------------------------------
    // Per (8 x 4 patch, part): the 32 cells' parts interleaved vector by
    // vector (layouts in pat_internal.h).  Fraction lists: hits counted per
    // cell, each block as long as the patch's longest part (fill in
    // k_adj_build).  Code lists: per (patch, detector block) the longest entry
    // count of the patch's cells sets the block's segment; the segments make
    // the patch's sequence, cut into G equal parts (fill in k_adj_seg).
    int64_t list_bytes = 0;
    if (use_lists) {
        const int S = frac_lists ? 3 : 1;     // 16-byte slots per vector of four entries
        const int G = LG;
        dp.adj_groups = G;                    // the fill kernels split lists into G parts
        std::vector<int> rep(tmpls.size(), -1);   // first instance of each geometry template
        for (int i = 0; i < n_inst; ++i)
            if (rep[inst_tmpl[i]] < 0) rep[inst_tmpl[i]] = i;
        for (size_t t = 0; t < tmpls.size(); ++t) {
            const int w = inst[rep[t]].n + 1;
            for (int i = 0; i < n_inst; ++i)
                if (inst_tmpl[i] == (int)t) inst[i].patches_x = (w + kPatchW - 1) / kPatchW;
        }
        if (cudaMemcpyAsync(base + o_inst, inst.data(), sizeof(InstDev) * inst.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            return PAT_ERR_CUDA;
        std::vector<int32_t> cnt_all;             // fraction lists: samples per cell
        std::vector<int64_t> tmpl_cnt_off(tmpls.size(), 0), tmpl_pbase_off(tmpls.size());
        std::vector<std::vector<int32_t>> part_len(tmpls.size());
        std::vector<int64_t> pbase_all;
        std::vector<int> nblk(tmpls.size(), 0);   // code lists: detector blocks per template
        int32_t* d_seg = nullptr;                 // code lists: per patch, segment starts + length (fill only)
        std::vector<int64_t> seg_off(tmpls.size() + 1, 0), slot0(tmpls.size() + 1, 0);
        int64_t slots_total = 0;   // 16-byte slots
        if (frac_lists) {
            std::vector<std::vector<int32_t>> counts(tmpls.size());
            int32_t* d_counts = nullptr;
            int64_t max_cells = 0;
            for (size_t t = 0; t < tmpls.size(); ++t)
                max_cells = std::max<int64_t>(max_cells, (int64_t)(inst[rep[t]].n + 1) * (inst[rep[t]].n + 1));
            if (dev_malloc(reinterpret_cast<void**>(&d_counts), sizeof(int32_t) * max_cells) != cudaSuccess) {
                cudaGetLastError();
                return PAT_ERR_OOM;
            }
            pat_status_t s = PAT_OK;
            for (size_t t = 0; t < tmpls.size() && s == PAT_OK; ++t) {
                const int i = rep[t];
                const int cells = (inst[i].n + 1) * (inst[i].n + 1);
                if (launch_adj_frac_build(dp, i, inst[i].n, d_counts, nullptr, nullptr, st) != cudaSuccess)
                    s = PAT_ERR_CUDA;
                counts[t].resize(cells);
                if (s == PAT_OK && cudaMemcpyAsync(counts[t].data(), d_counts, sizeof(int32_t) * cells,
                                                   cudaMemcpyDeviceToHost, st) != cudaSuccess)
                    s = PAT_ERR_CUDA;
                if (s == PAT_OK && cudaStreamSynchronize(st) != cudaSuccess) s = PAT_ERR_CUDA;
            }
            cudaFree(d_counts);
            if (s != PAT_OK) return s;
            for (size_t t = 0; t < tmpls.size(); ++t) {
                const int n = inst[rep[t]].n, w = n + 1;
                const int pw = (w + kPatchW - 1) / kPatchW, ph = (w + kPatchH - 1) / kPatchH;
                tmpl_cnt_off[t] = (int64_t)cnt_all.size();
                cnt_all.insert(cnt_all.end(), counts[t].begin(), counts[t].end());
                tmpl_pbase_off[t] = (int64_t)pbase_all.size();
                part_len[t].assign((size_t)pw * ph * G, 0);
                for (int py = 0; py < ph; ++py)
                    for (int px = 0; px < pw; ++px)
                        for (int g = 0; g < G; ++g) {
                            int V = 0;
                            for (int dy = 0; dy < kPatchH; ++dy)
                                for (int dx = 0; dx < kPatchW; ++dx) {
                                    const int cxa = px * kPatchW + dx, cya = py * kPatchH + dy;   // cell + 1
                                    if (cxa >= w || cya >= w) continue;
                                    const int nv = (counts[t][(size_t)cya * w + cxa] + 3) >> 2;
                                    const int v0 = (int)((int64_t)g * nv / G), v1 = (int)((int64_t)(g + 1) * nv / G);
                                    V = std::max(V, v1 - v0);
                                }
                            part_len[t][((size_t)py * pw + px) * G + g] = V;
                            pbase_all.push_back(slots_total);
                            slots_total += (int64_t)V * S * kWarp;
                        }
            }
        } else {
            // longest entry count per (patch, detector block), per template
            for (size_t t = 0; t < tmpls.size(); ++t) {
                const int w = inst[rep[t]].n + 1;
                const int64_t patches_t = (int64_t)((w + kPatchW - 1) / kPatchW) * ((w + kPatchH - 1) / kPatchH);
                nblk[t] = (inst[rep[t]].n_det + jblock - 1) / jblock;
                seg_off[t + 1] = seg_off[t] + patches_t * (nblk[t] + 1);
            }
            if (dev_malloc(reinterpret_cast<void**>(&d_seg), sizeof(int32_t) * std::max<int64_t>(seg_off.back(), 1)) !=
                cudaSuccess) {
                cudaGetLastError();
                return PAT_ERR_OOM;
            }
            pat_status_t s = PAT_OK;
            if (cudaMemsetAsync(d_seg, 0, sizeof(int32_t) * seg_off.back(), st) != cudaSuccess) s = PAT_ERR_CUDA;
            for (size_t t = 0; t < tmpls.size() && s == PAT_OK; ++t) {
                const int i = rep[t];
                if (launch_adj_seg(dp, i, inst[i].n, list_mode == 4, jblock, nblk[t], d_seg + seg_off[t], nullptr,
                                   nullptr, st) != cudaSuccess)
                    s = PAT_ERR_CUDA;
            }
            std::vector<int32_t> seg_host(seg_off.back());
            if (s == PAT_OK && cudaMemcpyAsync(seg_host.data(), d_seg, sizeof(int32_t) * seg_host.size(),
                                               cudaMemcpyDeviceToHost, st) != cudaSuccess)
                s = PAT_ERR_CUDA;
            if (s == PAT_OK && cudaStreamSynchronize(st) != cudaSuccess) s = PAT_ERR_CUDA;
            // segment starts, each patch's length in vectors, and the parts
            for (size_t t = 0; t < tmpls.size() && s == PAT_OK; ++t) {
                const int w = inst[rep[t]].n + 1;
                const int pw = (w + kPatchW - 1) / kPatchW, ph = (w + kPatchH - 1) / kPatchH;
                const int nb = nblk[t];
                tmpl_pbase_off[t] = (int64_t)pbase_all.size();
                slot0[t] = slots_total;
                part_len[t].assign((size_t)pw * ph * G, 0);
                for (int64_t pi = 0; pi < (int64_t)pw * ph; ++pi) {
                    int32_t* sp = seg_host.data() + seg_off[t] + pi * (nb + 1);
                    int64_t start = 0;
                    for (int b = 0; b < nb; ++b) {
                        const int32_t len = sp[b];
                        sp[b] = (int32_t)start;
                        start += len;
                    }
                    if (start > INT32_MAX - 3) s = PAT_ERR_UNSUPPORTED;
                    const int nv = (int)((start + 3) >> 2);
                    sp[nb] = nv;
                    for (int g = 0; g < G; ++g) {
                        const int V = (int)((int64_t)(g + 1) * nv / G) - (int)((int64_t)g * nv / G);
                        part_len[t][(size_t)pi * G + g] = V;
                        pbase_all.push_back(slots_total);
                        slots_total += (int64_t)V * kWarp;
                    }
                }
            }
            slot0[tmpls.size()] = slots_total;
            if (s == PAT_OK && cudaMemcpyAsync(d_seg, seg_host.data(), sizeof(int32_t) * seg_host.size(),
                                               cudaMemcpyHostToDevice, st) != cudaSuccess)
                s = PAT_ERR_CUDA;
            if (s != PAT_OK) {
                cudaStreamSynchronize(st);
                cudaFree(d_seg);
                return s;
            }
        }
        pbase_all.push_back(slots_total);   // end of the last block
        // work items: (patch, part) with their block and length
        std::vector<ListItem> li;
        for (int i = 0; i < n_inst; ++i) {
            const int t = inst_tmpl[i];
            const int n = inst[i].n, w = n + 1;
            const int pw = (w + kPatchW - 1) / kPatchW, ph = (w + kPatchH - 1) / kPatchH;
            for (int py = 0; py < ph; ++py)
                for (int px = 0; px < pw; ++px)
                    for (int g = 0; g < G; ++g) {
                        const size_t pi = ((size_t)py * pw + px) * G + g;
                        const int32_t V = part_len[t][pi];
                        if (V > 0)
                            li.push_back(ListItem{pbase_all[tmpl_pbase_off[t] + pi], V, i, g, px * kPatchW - 1,
                                                  py * kPatchH - 1, 0});
                    }
        }
        // static schedule: items to the warps of the launch, longest first to
        // the least loaded warp (a vector costs the same everywhere; an item
        // start costs about one vector more), then each warp's items in
        // (instance, patch) order
        const int lbps = adj_list_blocks_per_sm(list_lm);
        if (lbps < 1) {
            if (d_seg) {
                cudaStreamSynchronize(st);
                cudaFree(d_seg);
            }
            return PAT_ERR_UNSUPPORTED;
        }
        const int lblocks = (int)std::max<int64_t>(
            1, std::min<int64_t>((int64_t)lbps * P.num_sms, ((int64_t)li.size() + 7) / 8));
        const int n_warps = lblocks * 8;
        std::vector<int32_t> warp_items(n_warps + 1, 0);
        std::vector<ListItem> sched(li.size());
        int32_t n_tail = 0;
        {
            std::vector<int32_t> order(li.size());
            for (size_t k = 0; k < li.size(); ++k) order[k] = (int32_t)k;
            std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return li[a].nk > li[b].nk; });
            // the smallest items, about kListTailShare of the work, form a shared
            // queue that the warps drain after their own items: it absorbs the
            // run-time spread the static cost model does not see (cache
            // behaviour differs between regions of the image)
            int64_t total = 0;
            for (const ListItem& x : li) total += x.nk + 1;
            size_t n_static = order.size();
            for (int64_t tail_cost = 0; n_static > 0;) {
                const int64_t c = li[order[n_static - 1]].nk + 1;
                if ((double)(tail_cost + c) > kListTailShare * (double)total) break;
                tail_cost += c;
                --n_static;
            }
            n_tail = (int32_t)(order.size() - n_static);
            using Load = std::pair<int64_t, int32_t>;   // (cost, warp)
            std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
            for (int wv = 0; wv < n_warps; ++wv) heap.push({0, wv});
            std::vector<int32_t> owner(li.size(), -1);
            for (size_t r = 0; r < n_static; ++r) {
                const int32_t k = order[r];
                Load l = heap.top();
                heap.pop();
                owner[k] = l.second;
                l.first += li[k].nk + 1;
                heap.push(l);
            }
            for (size_t k = 0; k < li.size(); ++k)
                if (owner[k] >= 0) ++warp_items[owner[k] + 1];
            for (int wv = 0; wv < n_warps; ++wv) warp_items[wv + 1] += warp_items[wv];
            std::vector<int32_t> fill(warp_items.begin(), warp_items.end() - 1);
            for (size_t k = 0; k < li.size(); ++k)   // (li is in patch order)
                if (owner[k] >= 0) sched[fill[owner[k]]++] = li[k];
            for (size_t r = n_static; r < order.size(); ++r) sched[n_static + (r - n_static)] = li[order[r]];
        }
        const size_t b_pbase = sizeof(int64_t) * std::max<size_t>(pbase_all.size(), 1);
        const size_t b_cnt = sizeof(int32_t) * std::max<size_t>(cnt_all.size(), 1);
        const size_t b_items = sizeof(ListItem) * std::max<size_t>(sched.size(), 1);
        const size_t b_witems = sizeof(int32_t) * warp_items.size();
        const size_t b_codes = 16 * (size_t)std::max<int64_t>(slots_total, 1);
        const size_t o_cnt_l = align(b_pbase), o_items_l = align(o_cnt_l + b_cnt);
        const size_t o_witems_l = align(o_items_l + b_items);
        const size_t o_codes_l = align(o_witems_l + b_witems);
        list_bytes = (int64_t)(o_codes_l + b_codes);
        auto drop_seg = [&]() {   // (the segment table is only needed by the fill)
            if (d_seg) {
                cudaStreamSynchronize(st);
                cudaFree(d_seg);
                d_seg = nullptr;
            }
        };
        if (dev_malloc(&P.d_lists, list_bytes) != cudaSuccess) {
            P.d_lists = nullptr;
            cudaGetLastError();
            drop_seg();
            return PAT_ERR_OOM;
        }
        unsigned char* lb = static_cast<unsigned char*>(P.d_lists);
        uint32_t* codes = reinterpret_cast<uint32_t*>(lb + o_codes_l);
        if (cudaMemcpyAsync(lb, pbase_all.data(), sizeof(int64_t) * pbase_all.size(), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            (!cnt_all.empty() &&
             cudaMemcpyAsync(lb + o_cnt_l, cnt_all.data(), sizeof(int32_t) * cnt_all.size(), cudaMemcpyHostToDevice,
                             st) != cudaSuccess) ||
            (!sched.empty() && cudaMemcpyAsync(lb + o_items_l, sched.data(), sizeof(ListItem) * sched.size(),
                                               cudaMemcpyHostToDevice, st) != cudaSuccess) ||
            cudaMemcpyAsync(lb + o_witems_l, warp_items.data(), b_witems, cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemsetAsync(codes, 0, b_codes, st) != cudaSuccess) {
            drop_seg();
            return PAT_ERR_CUDA;
        }
        dp.list_base = reinterpret_cast<const int64_t*>(lb);
        dp.cell_cnt = frac_lists ? reinterpret_cast<const int32_t*>(lb + o_cnt_l) : nullptr;
        dp.list_items = reinterpret_cast<const ListItem*>(lb + o_items_l);
        dp.warp_items = reinterpret_cast<const int32_t*>(lb + o_witems_l);
        dp.codes = codes;
        dp.n_code_vecs = (int64_t)(b_codes / 16);
        for (int i = 0; i < n_inst; ++i) {
            inst[i].list_off = tmpl_cnt_off[inst_tmpl[i]];
            inst[i].pbase_off = tmpl_pbase_off[inst_tmpl[i]];
        }
        if (cudaMemcpyAsync(base + o_inst, inst.data(), sizeof(InstDev) * inst.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
            drop_seg();
            return PAT_ERR_CUDA;
        }
        // fill the lists (same enumeration, same order)
        for (size_t t = 0; t < tmpls.size(); ++t) {
            const int i = rep[t];
            cudaError_t e;
            if (frac_lists) {
                e = launch_adj_frac_build(dp, i, inst[i].n, const_cast<int32_t*>(dp.cell_cnt) + tmpl_cnt_off[t],
                                          dp.list_base + tmpl_pbase_off[t], codes, st);
            } else {
                // null codes (row 0, the always-zero column m_pitch - 1) everywhere first
                const int64_t s0 = slot0[t], s1 = slot0[t + 1];
                e = launch_fill_u32(codes + s0 * 4, (s1 - s0) * 4, (uint32_t)inst[i].m_pitch - 1u, st);
                if (e == cudaSuccess)
                    e = launch_adj_seg(dp, i, inst[i].n, list_mode == 4, jblock, nblk[t], d_seg + seg_off[t],
                                       dp.list_base + tmpl_pbase_off[t], codes, st);
            }
            if (e != cudaSuccess) {
                drop_seg();
                return PAT_ERR_CUDA;
            }
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            drop_seg();
            return PAT_ERR_CUDA;
        }
        drop_seg();
        dp.n_list_items = (int)li.size();
        dp.n_tail_items = n_tail;
        dp.list_tail0 = (int)li.size() - n_tail;
        dp.adj_mode = list_mode;
        dp.adj_jblock = jblock;
        dp.cell_blocks = lblocks;
    }

    // ---- info -------------------------------------------------------------
    pat_plan_info_t& I = P.info;
    std::memset(&I, 0, sizeof(I));
    I.n_instances = n_inst;
    I.device = dev;
    I.f_elems = P.f_offsets[n_inst];
    I.g_elems = P.g_offsets[n_inst];
    I.samples = (int64_t)count;
    I.sample_slots = samples_slots;
    I.time_macs = time_macs;
    I.work_units = (int64_t)units.size();
    I.device_bytes = (int64_t)P.tables_bytes + (int64_t)sizeof(float) * P.work_floats;
    I.m_lanes = ml;
    I.q_piece = qpiece;
    I.band_rows = 0;
    I.tile_cols = 0;
    for (auto& T : tmpls)
        for (auto& t : T.tiles) {
            I.band_rows = std::max(I.band_rows, t.y1 - t.y0);
            I.tile_cols = std::max(I.tile_cols, t.x1 - t.x0);
        }
    I.adj_groups = dp.adj_groups;
    I.adj_mode = dp.adj_mode == 0 ? 2 : dp.adj_mode;
    I.abel_split_fwd = dp.abel_cluster_fwd;
    I.abel_split_adj = dp.abel_cluster_adj;
    I.time_pair = dp.time_chunks > 0 ? 1 : 0;
    I.adj_jblock = dp.adj_jblock;
    I.list_bytes = list_bytes;
    I.device_bytes += list_bytes;
    I.bands_max = tiles_max;
    return PAT_OK;
}

namespace {
std::atomic<int32_t> g_alloc_fail{-1};   // see set_alloc_failure
} // namespace

void set_alloc_failure(int32_t n) { g_alloc_fail.store(n < 0 ? -1 : n); }

cudaError_t dev_malloc(void** p, size_t bytes)
{
    int32_t k = g_alloc_fail.load();
    while (k >= 0 && !g_alloc_fail.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

void free_plan_memory(Plan& P)
{
    for (auto& v : P.recorded)
        for (auto& e : v) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    for (auto e : P.event_pool) cudaEventDestroy(e);
    for (auto& v : P.recorded) v.clear();
    P.event_pool.clear();
    if (P.d_tables) cudaFree(P.d_tables);
    if (P.d_work) cudaFree(P.d_work);
    if (P.d_lists) cudaFree(P.d_lists);
    P.d_lists = nullptr;
    P.d_tables = nullptr;
    P.d_work = nullptr;
}

} // namespace patgpu
