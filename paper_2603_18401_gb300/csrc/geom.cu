// Geometry and per-keypoint preparation.
//
//   geometry_kernel   one block per pair: epipole e2 = null(F^T) (Algorithm 1)
//                     as the cross product of two columns of F, the key frame
//                     (angular or parallel) and zeroed level statistics.
//   prep_kernel       every reference keypoint: its angle seen from e2
//                     (Sec. 4.2, Eq. theta), its level (the octave of
//                     eps_j / ||p_j - e2||, i.e. of sin delta_j, Eq. delta), a
//                     27-bit sort key; every query: its epipolar line
//                     l_i = F p~_i^1 (Sec. 3) in FP64, the line's angle alpha_i
//                     (Sec. 4.2, reduced mod pi) and the FP32 line used by the
//                     pre-test.
//   intervals_kernel  the paper's (theta_j, delta_j) in FP64 for inspection.
//
// Angles are measured in a frame turned so that the image centre lies at
// angle 0 as seen from the epipole, and reduced to [-pi/2, pi/2) by flipping
// the direction vector (exact) rather than by adding pi (rounded).
#include <math.h>

#include "egm_internal.cuh"

namespace egm {

namespace {

__device__ __forceinline__ void set_status(uint32_t *st, uint32_t bit) { atomicOr(st, bit); }

__device__ __forceinline__ void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__global__ void geometry_kernel(Launch L) {
    const int p = blockIdx.x;
    const PairDesc &P = L.pairs[p];
    PairGeom &G = L.geom[p];
    const int t = threadIdx.x;
    if (t < kLevels) {
        G.cnt[t] = 0u;
        G.smax[t] = 0u;
        G.dmin[t] = 0x7f800000u;  // +inf
        G.tmax[t] = 0u;
    }
    if (t != 0) return;

    double F[9];
    bool finite = true;
    double fn2 = 0.0;
    for (int k = 0; k < 9; k++) {
        F[k] = P.F[k];
        finite &= isfinite(F[k]);
        fn2 += F[k] * F[k];
    }
    const double W = (double)P.width, H = (double)P.height;
    const double cx = 0.5 * W, cy = 0.5 * H;
    // FP64 is scarce on this GPU: the range / mode decisions below only steer
    // efficiency (keys are clamped into any range), so they use FP32 maths on
    // FP64-computed offsets.
    const double diag = (double)hypotf((float)W, (float)H);
    G.cx = cx;
    G.cy = cy;

    // e2 is orthogonal to every column of F (F^T e2 = 0): take the cross
    // product of the two columns with the largest cross-product norm.
    double col[3][3] = {{F[0], F[3], F[6]}, {F[1], F[4], F[7]}, {F[2], F[5], F[8]}};
    double cr[3][3];
    cross3(col[0], col[1], cr[0]);
    cross3(col[0], col[2], cr[1]);
    cross3(col[1], col[2], cr[2]);
    int kb = 0;
    double nb = -1.0;
    for (int k = 0; k < 3; k++) {
        double nk = cr[k][0] * cr[k][0] + cr[k][1] * cr[k][1] + cr[k][2] * cr[k][2];
        if (nk > nb) { nb = nk; kb = k; }
    }
    bool degenerate = !finite || !(fn2 > 0.0) || !(nb > 1e-26 * fn2 * fn2);
    if (!finite) set_status(L.status, kStNan);
    else if (degenerate) set_status(L.status, kStDegenerateF);

    double ex = 1.0, ey = 0.0, ew = 0.0;
    if (!degenerate) {
        double s = 1.0 / sqrt(nb);
        ex = cr[kb][0] * s;
        ey = cr[kb][1] * s;
        ew = cr[kb][2] * s;
        if (ew < 0.0 || (ew == 0.0 && (ex < 0.0 || (ex == 0.0 && ey < 0.0)))) {
            ex = -ex; ey = -ey; ew = -ew;
        }
    }
    G.ex = ex;
    G.ey = ey;
    G.ew = ew;

    bool parallel = true;
    double xe = 0.0, ye = 0.0, D = INFINITY;
    if (!degenerate && ew != 0.0) {
        xe = ex / ew;
        ye = ey / ew;
        D = (double)hypotf((float)(xe - cx), (float)(ye - cy));
        parallel = !(D <= 1e6 * diag);
    }
    G.xe = xe;
    G.ye = ye;
    const double corners[4][2] = {{0.0, 0.0}, {W, 0.0}, {0.0, H}, {W, H}};
    const double eps_ref = P.eps2 ? 1.0 : (P.eps_scalar > 0.0 ? P.eps_scalar : 1.0);

    if (parallel) {
        // All lines (nearly) parallel to u, the direction of the epipole.
        double ux = 1.0, uy = 0.0;
        if (!degenerate) {
            double vx = ex - cx * ew, vy = ey - cy * ew;
            double nv = sqrt(vx * vx + vy * vy);
            if (nv > 0.0) { ux = vx / nv; uy = vy / nv; }
        }
        G.mode = kModeParallel;
        G.ux = ux;
        G.uy = uy;
        double nx = -uy, ny = ux, lo = INFINITY, hi = -INFINITY;
        for (int k = 0; k < 4; k++) {
            double s = nx * (corners[k][0] - cx) + ny * (corners[k][1] - cy);
            lo = fmin(lo, s);
            hi = fmax(hi, s);
        }
        double margin = 0.01 * (hi - lo) + 1.0;
        G.kmin = (float)(lo - margin);
        G.kscale = (float)((double)kQMax / (hi - lo + 2.0 * margin));
        G.level_base = ilogb(eps_ref) - 8;
    } else {
        double vx = cx - xe, vy = cy - ye, nv = sqrt(vx * vx + vy * vy);
        double ux = 1.0, uy = 0.0;
        if (nv > 1e-9 * diag) { ux = vx / nv; uy = vy / nv; }
        G.mode = kModeAngular;
        G.ux = ux;
        G.uy = uy;
        double lo = INFINITY, hi = -INFINITY;
        for (int k = 0; k < 4; k++) {
            double wx = corners[k][0] - xe, wy = corners[k][1] - ye;
            double px = wx * ux + wy * uy, py = ux * wy - uy * wx;
            double a = (double)atan2f((float)py, (float)px);
            lo = fmin(lo, a);
            hi = fmax(hi, a);
        }
        double mx = 0.02 * diag;
        bool inside = xe >= -mx && xe <= W + mx && ye >= -mx && ye <= H + mx;
        if (inside || hi > 1.3 || lo < -1.3) {
            G.kmin = -kHalfPiF;
            G.kscale = (float)((double)kQMax / M_PI);
        } else {
            double margin = 0.02 * (hi - lo);
            G.kmin = (float)(lo - margin);
            G.kscale = (float)((double)kQMax / (hi - lo + 2.0 * margin));
        }
        // distance from e2 to the image rectangle
        double dx = fmax(fmax(-xe, xe - W), 0.0), dy = fmax(fmax(-ye, ye - H), 0.0);
        double dr = (double)hypotf((float)dx, (float)dy);
        G.level_base = ilogb(fmax(dr, 2.0 * eps_ref) / eps_ref) - 1;
    }
}

__global__ void __launch_bounds__(256) prep_kernel(Launch L) {
    const int64_t total = L.nr + L.nq;
    const int lane = threadIdx.x & 31;
    for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x; g0 < total; g0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = g0 + threadIdx.x;
        const bool valid = g < total;
        const bool is_ref = g < L.nr;
        uint32_t group = 0xffffffffu;
        uint32_t s_bits = 0, d_bits = 0x7f800000u, t_bits = 0;
        int p = 0;
        if (valid && is_ref) {
            p = pair_of(L.r_offs, L.npairs, g);
            const PairDesc &P = L.pairs[p];
            const PairGeom &G = L.geom[p];
            const int64_t j = g - P.r_off;
            const double x = P.xy2[2 * j], y = P.xy2[2 * j + 1];
            const double eps = P.eps2 ? P.eps2[j] : P.eps_scalar;
            if (!(isfinite(x) && isfinite(y) && isfinite(eps))) set_status(L.status, kStNan);
            else if (!(eps > 0.0)) set_status(L.status, kStArg);
            const float epsf = (float)eps;
            int level;
            float key;
            if (G.mode == kModeAngular) {
                const double vx = x - G.xe, vy = y - G.ye;
                double px = vx * G.ux + vy * G.uy;
                double py = G.ux * vy - G.uy * vx;
                if (px < 0.0 || (px == 0.0 && py > 0.0)) { px = -px; py = -py; }
                key = atan2f((float)py, (float)px);
                const float d = hypotf((float)vx, (float)vy);
                const float ratio = d / epsf;
                if (!(ratio >= 2.0f)) {
                    level = 0;
                } else {
                    level = ilogbf(ratio) - G.level_base;
                    level = level < 1 ? 1 : (level > kLevels - 1 ? kLevels - 1 : level);
                }
                float s = d > 0.0f ? epsf / d : INFINITY;
                s_bits = __float_as_uint(s * 1.000001f);
                d_bits = __float_as_uint(d * 0.999999f);
            } else {
                const double px = x - G.cx, py = y - G.cy;
                const double sN = -G.uy * px + G.ux * py;
                const double tU = G.ux * px + G.uy * py;
                key = (float)sN;
                level = ilogbf(epsf) - G.level_base;
                level = level < 1 ? 1 : (level > kLevels - 1 ? kLevels - 1 : level);
                s_bits = __float_as_uint(epsf * 1.000001f);
                t_bits = __float_as_uint((float)fabs(tU) * 1.000001f + 1e-3f);
            }
            if (!isfinite(key)) key = 0.0f;
            const uint32_t q = qmap(key, G.kmin, G.kscale);
            L.key_a[g] = ((uint32_t)level << kQBits) | q;
            L.val_a[g] = (uint32_t)j;
            group = (uint32_t)p * kLevels + (uint32_t)level;
        } else if (valid) {
            const int64_t gq = g - L.nr;
            p = pair_of(L.q_offs, L.npairs, gq);
            const PairDesc &P = L.pairs[p];
            const PairGeom &G = L.geom[p];
            const int64_t i = gq - P.q_off;
            const double x1 = P.xy1[2 * i], y1 = P.xy1[2 * i + 1];
            QueryRec r;
            r.flags = 0;
            r.pad = 0;
            r.A = r.B = r.C = r.key = r.aux0 = r.aux1 = 0.0f;
            if (!(isfinite(x1) && isfinite(y1))) set_status(L.status, kStNan);
            double a, b, c;
            exact_line(P.F, x1, y1, a, b, c);
            const double N = exact_norm(a, b);
            if (!(N > 0.0) || !isfinite(N) || !isfinite(c)) {
                r.flags = EGM_FLAG_DEGENERATE_LINE;
            } else {
                const double inv = 1.0 / N;
                double A = a * inv, B = b * inv, C = (a * G.cx + b * G.cy + c) * inv;
                if (G.mode == kModeAngular) {
                    const double tx = B, ty = -A;  // line direction
                    double px = tx * G.ux + ty * G.uy;
                    double py = G.ux * ty - G.uy * tx;
                    if (px < 0.0 || (px == 0.0 && py > 0.0)) { px = -px; py = -py; }
                    r.key = atan2f((float)py, (float)px);
                    // distance of the computed epipole from the line, plus a
                    // bound on its FP64 rounding error
                    const double ta = a * G.xe, tb = b * G.ye;
                    const double rr = fabs(ta + tb + c) * inv;
                    const double err = 4.5e-16 * (fabs(ta) + fabs(tb) + fabs(c)) * inv;
                    r.aux0 = __double2float_ru((rr + err) * (1.0 + 1e-12) + 1e-9);
                } else {
                    const double nx = -G.uy, ny = G.ux;
                    double cphi = A * nx + B * ny;
                    if (cphi < 0.0) { A = -A; B = -B; C = -C; cphi = -cphi; }
                    const double sphi = fabs(A * G.ux + B * G.uy);
                    r.aux0 = __double2float_rd(cphi);
                    r.aux1 = __double2float_ru(sphi);
                    r.key = cphi > 0.5 ? (float)(-C / cphi) : 0.0f;
                }
                r.A = (float)A;
                r.B = (float)B;
                r.C = (float)C;
                if (!isfinite(r.C) || !isfinite(r.key)) r.flags = EGM_FLAG_DEGENERATE_LINE;
            }
            L.qrec[gq] = r;
        }
        // warp-aggregated level statistics
        const uint32_t peers = __match_any_sync(0xffffffffu, group);
        const uint32_t smax = __reduce_max_sync(peers, s_bits);
        const uint32_t dmin = __reduce_min_sync(peers, d_bits);
        const uint32_t tmax = __reduce_max_sync(peers, t_bits);
        if (group != 0xffffffffu && lane == __ffs(peers) - 1) {
            const int pp = (int)(group / kLevels), lv = (int)(group % kLevels);
            PairGeom &G = L.geom[pp];
            atomicAdd(&G.cnt[lv], (uint32_t)__popc(peers));
            atomicMax(&G.smax[lv], smax);
            atomicMin(&G.dmin[lv], dmin);
            atomicMax(&G.tmax[lv], tmax);
        }
    }
}

__global__ void intervals_kernel(Launch L, double *theta, double *delta, double *e3, int32_t *mode) {
    const PairDesc &P = L.pairs[0];
    const PairGeom &G = L.geom[0];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) {
        if (e3) { e3[0] = G.ex; e3[1] = G.ey; e3[2] = G.ew; }
        if (mode) mode[0] = G.mode;
    }
    if (j >= P.n) return;
    double th = NAN, de = NAN;
    if (G.mode == kModeAngular) {
        const double dx = P.xy2[2 * j] - G.xe, dy = P.xy2[2 * j + 1] - G.ye;
        const double eps = P.eps2 ? P.eps2[j] : P.eps_scalar;
        const double d = hypot(dx, dy);
        th = atan2(dy, dx);
        if (th < 0.0) th += M_PI;
        if (th >= M_PI) th -= M_PI;
        de = d <= eps ? 0.5 * M_PI : asin(eps / d);
    }
    if (theta) theta[j] = th;
    if (delta) delta[j] = de;
}

}  // namespace

cudaError_t launch_geometry(const Launch &L, cudaStream_t s) {
    geometry_kernel<<<L.npairs, 32, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_prep(const Launch &L, cudaStream_t s) {
    const int64_t total = L.nr + L.nq;
    if (total == 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    prep_kernel<<<(int)blocks, 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_intervals(const Launch &L, double *theta, double *delta, double *e3, int32_t *mode,
                             cudaStream_t s) {
    int64_t n = L.nr;
    int blocks = (int)((n + 255) / 256);
    if (blocks < 1) blocks = 1;
    intervals_kernel<<<blocks, 256, 0, s>>>(L, theta, delta, e3, mode);
    return cudaGetLastError();
}

}  // namespace egm
