// Geometry and per-keypoint preparation.
//
//   geometry_kernel   one warp per pair: epipole e2 = null(F^T) (Algorithm 1)
//                     as the cross product of two columns of F, the key frame
//                     (angular or parallel) and zeroed level statistics.
//   prep_kernel       every reference keypoint: its angle seen from e2
//                     (Sec. 4.2, Eq. theta), its level (the octave of
//                     eps_j / ||p_j - e2||, i.e. of sin delta_j, Eq. delta) and
//                     a 27-bit sort key; every query: its epipolar line
//                     l_i = F p~_i^1 (Sec. 3), the line's angle alpha_i
//                     (Sec. 4.2, reduced mod pi) and the FP32 line of the
//                     pre-test, with bounds on every rounding error.
//   intervals_kernel  the paper's (theta_j, delta_j) in FP64 for inspection.
//
// FP64 is scarce on GB300 (about 1/64 of the FP32 rate), so only what needs
// it runs in FP64: the epipole, the query line (FMA form) and two dot
// products per query.  The angular frame is turned so that the image centre
// c lies at angle 0 seen from the epipole e; with E = e - c and u the unit
// vector towards c, the exact decomposition
//     p - e  =  (|E| + u.(p - c),  u x (p - c) + kappa),   kappa = -u x E,
// lets every reference be keyed in FP32 even when e is 1e10 px away: kappa
// (computed once in FP64) absorbs the rounding of u.  A direction is reduced
// mod pi by flipping the vector (exact), never by adding pi (rounded).
#include <math.h>

#include "egm_internal.cuh"

namespace egm {

namespace {

__device__ __forceinline__ void set_status(uint32_t *st, uint32_t bit) { atomicOr(st, bit); }

// The hardware conversion for the values d2f leaves to it (kept out of line,
// so that the common case issues no FP64-pipe instruction).
__device__ __noinline__ float d2f_other(double d) { return __double2float_rn(d); }

// double -> float rounded to nearest, ties to even, on the integer pipes (the
// IEEE 754 conversion: keep the sign, rebias the exponent, keep the top 23
// fraction bits and round on the 29 dropped ones; a carry out of the
// fraction moves into the exponent, and from the largest finite float to
// infinity, as rounding to nearest requires).  Only results that are normal
// floats before rounding take this path: zeros, subnormals, values above the
// float range and non-finite values take the hardware conversion.  GB300
// issues FP64-pipe instructions, conversions included, at a small fraction of
// its integer rate.
__device__ __forceinline__ float d2f(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const uint32_t e = (hi >> 20) & 0x7ffu;
    if (e - 897u > 253u) return d2f_other(d);  // float exponent field (e - 896) outside 1..254
    uint32_t f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1fffffffu;
    f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
}

// |(x, y)| within a few ulps: the square root of the FMA sum of squares
// where that sum is a normal float far from overflow (a component lost to
// underflow then changes the norm by far less than an ulp), hypotf elsewhere.
__device__ __forceinline__ float norm2f(float x, float y) {
    const float s = fmaf(x, x, y * y);
    if (s >= 1e-30f && s <= 1e30f) return sqrtf(s);
    return hypotf(x, y);
}

__device__ __forceinline__ float fold_atan2(float px, float py) {
    if (px < 0.0f || (px == 0.0f && py > 0.0f)) { px = -px; py = -py; }
    return atan2f(py, px);
}

// The geometry kernel reads only its parameters (or a pair table uploaded
// before it) and writes this call's half of the double-buffered pair table,
// offsets and geometry, which the previous call no longer reads: it computes
// while the previous call's last kernel runs and waits for that kernel only
// before it ends, so that the kernels after it see the previous call done.
__global__ void __launch_bounds__(32) geometry_kernel(Launch L) {
    pdl_trigger();
    const int p = blockIdx.x;
    const int lane = threadIdx.x;
    if (L.inl_use) {
        // one pair: write its plan for the later kernels
        if (lane == 0) {
            *const_cast<PairDesc *>(L.pairs) = L.inl;
            int64_t *qo = const_cast<int64_t *>(L.q_offs), *ro = const_cast<int64_t *>(L.r_offs);
            qo[0] = 0;
            qo[1] = L.inl.m;
            ro[0] = 0;
            ro[1] = L.inl.n;
            if (L.tile_offs) {
                int64_t *to = const_cast<int64_t *>(L.tile_offs);
                to[0] = 0;
                to[1] = L.ntiles;
            }
        }
        if (L.tile_seq)
            for (int64_t t = lane; t < L.ntiles; t += 32) const_cast<int2 *>(L.tile_seq)[t] = make_int2((int)t, 0);
    }
    const PairDesc &P = L.inl_use ? L.inl : L.pairs[p];
    PairGeom &G = L.geom[p];
    G.cnt[lane] = 0u;
    G.smax[lane] = 0u;
    G.dmin[lane] = 0x7f800000u;  // +inf
    G.tmax[lane] = 0u;
    if (lane == 0) {
        G.qa0max = 0u;
        G.qa0min = 0x7f800000u;
        G.qa1max = 0u;
        G.qkabs = 0u;
    }

    // F^T e2 = 0: e2 is orthogonal to every column of F.  Lanes 0..2 form the
    // three column cross products; the largest one is the epipole.
    const double fv = lane < 9 ? P.F[lane] : 0.0;
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; k++) F[k] = __shfl_sync(0xffffffffu, fv, k);
    const bool finite = __all_sync(0xffffffffu, isfinite(fv));
    double fn2 = 0.0;
#pragma unroll
    for (int k = 0; k < 9; k++) fn2 = fma(F[k], F[k], fn2);
    // column pairs (0,1) (0,2) (1,2), picked by selects (an index that depends
    // on the lane would move F to local memory)
    const bool a1 = lane == 2, b1 = lane == 0;
    const double ax = a1 ? F[1] : F[0], ay = a1 ? F[4] : F[3], az = a1 ? F[7] : F[6];
    const double bx = b1 ? F[1] : F[2], by = b1 ? F[4] : F[5], bz = b1 ? F[7] : F[8];
    double crx = fma(ay, bz, -az * by), cry = fma(az, bx, -ax * bz), crz = fma(ax, by, -ay * bx);
    double nk = lane < 3 ? fma(crx, crx, fma(cry, cry, crz * crz)) : -1.0;
    int best = lane;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        const double on = __shfl_xor_sync(0xffffffffu, nk, o);
        const int ob = __shfl_xor_sync(0xffffffffu, best, o);
        if (on > nk || (on == nk && ob < best)) { nk = on; best = ob; }
    }
    crx = __shfl_sync(0xffffffffu, crx, best);
    cry = __shfl_sync(0xffffffffu, cry, best);
    crz = __shfl_sync(0xffffffffu, crz, best);
    const bool degenerate = !finite || !(fn2 > 0.0) || !(nk > 1e-26 * fn2 * fn2);

    const double W = (double)P.width, H = (double)P.height;
    const double cx = 0.5 * W, cy = 0.5 * H;
    const float diag = hypotf((float)W, (float)H);
    double ex = 1.0, ey = 0.0, ew = 0.0;
    if (!degenerate) {
        const double s = 1.0 / sqrt(nk);
        ex = crx * s;
        ey = cry * s;
        ew = crz * s;
        if (ew < 0.0 || (ew == 0.0 && (ex < 0.0 || (ex == 0.0 && ey < 0.0)))) {
            ex = -ex; ey = -ey; ew = -ew;
        }
    }
    bool parallel = true;
    double xe = 0.0, ye = 0.0;
    double Ex = 0.0, Ey = 0.0;
    if (!degenerate && ew != 0.0) {
        const double iw = 1.0 / ew;
        xe = ex * iw;
        ye = ey * iw;
        Ex = xe - cx;
        Ey = ye - cy;
        parallel = !(hypotf((float)Ex, (float)Ey) <= 1e6f * diag);
    }
    // frame: FP32 unit vector u and, in angular mode, |E| and kappa
    float ux = 1.0f, uy = 0.0f, de = 0.0f, kappa = 0.0f;
    if (parallel) {
        if (!degenerate) {
            const double vx = ex - cx * ew, vy = ey - cy * ew;
            const float nv = hypotf((float)vx, (float)vy);
            if (nv > 0.0f) { ux = (float)vx / nv; uy = (float)vy / nv; }
        }
    } else {
        const double dE = sqrt(fma(Ex, Ex, Ey * Ey));
        if (dE > 1e-9 * (double)diag) {
            ux = (float)(-Ex / dE);
            uy = (float)(-Ey / dE);
        }
        de = (float)dE;
        // kappa = -(u x E) with the rounded u, in FP64
        kappa = (float)(-fma((double)ux, Ey, -(double)uy * Ex));
    }
    // key range from the image corners (lane k < 4), FP32
    const float qx = (lane & 1) ? (float)(W - cx) : (float)(-cx);
    const float qy = (lane & 2) ? (float)(H - cy) : (float)(-cy);
    float kv;
    if (parallel) kv = -uy * qx + ux * qy;
    else kv = fold_atan2(de + (ux * qx + uy * qy), (ux * qy - uy * qx) + kappa);
    float lo = lane < 4 ? kv : INFINITY, hi = lane < 4 ? kv : -INFINITY;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane < 9) G.Ff[lane] = (float)fv;
    // lanes 0..2: v_k = F_k xe + F_{3+k} ye + F_{6+k} (two roundings, each at
    // most 2^-53 of the terms' magnitudes), bounded above in FP32
    {
        const double f0 = __shfl_sync(0xffffffffu, fv, lane % 3), f1 = __shfl_sync(0xffffffffu, fv, lane % 3 + 3),
                     f2 = __shfl_sync(0xffffffffu, fv, lane % 3 + 6);
        float vb = 0.0f;
        if (!parallel) {
            const double v = fma(f0, xe, fma(f1, ye, f2));
            const double T = fabs(f0 * xe) + fabs(f1 * ye) + fabs(f2);
            vb = (float)(fabs(v) + 4.5e-16 * T) * 1.000001f;
        }
        if (lane < 3) G.vb[lane] = vb;
    }
    if (lane != 0) {
        pdl_wait();
        return;
    }
    if (!finite) set_status(L.status, kStNan);
    else if (degenerate) set_status(L.status, kStDegenerateF);
    G.ex = ex;
    G.ey = ey;
    G.ew = ew;
    G.xe = xe;
    G.ye = ye;
    G.cx = cx;
    G.cy = cy;
    G.cxf = (float)cx;
    G.cyf = (float)cy;
    G.xef = (float)xe;
    G.yef = (float)ye;
    G.ux = ux;
    G.uy = uy;
    G.de = de;
    G.kappa = kappa;
    const float eps_ref = P.eps2 ? 1.0f : (P.eps_scalar > 0.0 ? (float)P.eps_scalar : 1.0f);
    if (parallel) {
        G.mode = kModeParallel;
        const float margin = 0.01f * (hi - lo) + 1.0f;
        G.kmin = lo - margin;
        G.kscale = (float)kQMax / (hi - lo + 2.0f * margin);
        G.level_base = ilogbf(eps_ref) - 8;
    } else {
        G.mode = kModeAngular;
        const float mx = 0.02f * diag;
        const float fxe = (float)xe, fye = (float)ye;
        const bool inside = fxe >= -mx && fxe <= (float)W + mx && fye >= -mx && fye <= (float)H + mx;
        if (inside || hi > 1.3f || lo < -1.3f) {
            G.kmin = -kHalfPiF;
            G.kscale = (float)kQMax / kPiF;
        } else {
            const float margin = 0.02f * (hi - lo);
            G.kmin = lo - margin;
            G.kscale = (float)kQMax / (hi - lo + 2.0f * margin);
        }
        // distance from e2 to the image rectangle
        const float dx = fmaxf(fmaxf(-fxe, fxe - (float)W), 0.0f), dy = fmaxf(fmaxf(-fye, fye - (float)H), 0.0f);
        const float dr = hypotf(dx, dy);
        G.level_base = ilogbf(fmaxf(dr, 2.0f * eps_ref) / eps_ref) - 1;
    }
    pdl_wait();
}


// part: 0 every row; 1 the references (with the tables' zeroing and the
// level layout); 2 the queries (the banded form runs them beside part 1:
// nothing of either part reads the other's output)
__global__ void __launch_bounds__(256) prep_kernel(Launch L, int part) {
    pdl_begin();
    const int64_t total = L.nr + L.nq;
    const int64_t lo = part == 2 ? L.nr : 0, hi = part == 1 ? L.nr : total;
    const int lane = threadIdx.x & 31;
    __shared__ int64_t s_roffs[kSmemPairs + 1], s_qoffs[kSmemPairs + 1];
    // one pair (plan in the parameters): every row is pair 0, no offsets to load
    const bool one = L.inl_use != 0;
    const bool cached = one || (load_offsets(s_roffs, L.r_offs, L.npairs) && load_offsets(s_qoffs, L.q_offs, L.npairs));
    __syncthreads();
    // the bucket tables start from zero (the counting sort after this kernel fills them)
    if (part != 2)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.ntab / 4;
             i += (int64_t)gridDim.x * blockDim.x)
            reinterpret_cast<uint4 *>(L.tab)[i] = make_uint4(0, 0, 0, 0);
    for (int64_t g0 = lo + (int64_t)blockIdx.x * blockDim.x; g0 < hi; g0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = g0 + threadIdx.x;
        const bool valid = g < hi;
        const bool is_ref = g < L.nr;
        // the row's pair (the warp is converged here; a warp with no valid
        // row skips the lookup as a whole)
        int p = 0;
        if (!one) {
            if (cached) {
                if (g0 + (threadIdx.x & ~31) < hi) p = warp_pair(s_roffs, s_qoffs, L.npairs, L.nr, g);
            } else if (valid) {
                p = is_ref ? pair_of(L.r_offs, L.npairs, g) : pair_of(L.q_offs, L.npairs, g - L.nr);
            }
        }
        uint32_t group = 0xffffffffu;
        uint32_t s_bits = 0, d_bits = 0x7f800000u, t_bits = 0;
        uint32_t qgroup = 0xffffffffu, qa0 = 0u, qa1 = 0u, qk = 0u;
        if (valid && is_ref) {
            const PairView P = pair_view(L, p);
            const PairGeom &G = L.geom[p];
            const int64_t j = g - P.r_off;
            const double x = P.xy2[2 * j], y = P.xy2[2 * j + 1];
            const double eps = P.eps2 ? P.eps2[j] : P.eps_scalar;
            if (!(finite64(x) && finite64(y) && finite64(eps))) set_status(L.status, kStNan);
            else if (!positive64(eps)) set_status(L.status, kStArg);
            const float epsf = d2f(eps);
            const float xf = d2f(x - G.cx), yf = d2f(y - G.cy);
            // the reference's FP32 record, placed in its bucket by the sort
            L.rtmp[g] = make_float4(xf, yf, epsf, __uint_as_float((uint32_t)j));
            const float rr = norm2f(xf, yf);
            int level;
            float key;
            if (G.mode == kModeAngular) {
                const float px = G.de + (G.ux * xf + G.uy * yf);
                const float py = (G.ux * yf - G.uy * xf) + G.kappa;
                key = fold_atan2(px, py);
                const float d = norm2f(px, py);
                // the level only groups references (its statistics come from
                // its members): an approximate quotient serves
                const float ratio = __fdividef(d, epsf);
                if (!(ratio >= 2.0f)) {
                    level = 0;
                } else {
                    level = ilogbf(ratio) - G.level_base;
                    level = level < 1 ? 1 : (level > kLevels - 1 ? kLevels - 1 : level);
                }
                const float s = d > 0.0f ? epsf / d : INFINITY;
                s_bits = __float_as_uint(s * 1.000001f);
                d_bits = __float_as_uint(d * 0.999999f);
            } else {
                key = -G.uy * xf + G.ux * yf;
                level = ilogbf(epsf) - G.level_base;
                level = level < 1 ? 1 : (level > kLevels - 1 ? kLevels - 1 : level);
                s_bits = __float_as_uint(epsf * 1.000001f);
            }
            t_bits = __float_as_uint(rr * 1.000001f);
            if (!isfinite(key)) key = 0.0f;
            const uint32_t q = qmap(key, G.kmin, G.kscale);
            L.key_a[g] = ((uint32_t)level << kQBits) | q;
            group = (uint32_t)p * kLevels + (uint32_t)level;
        } else if (valid) {
            const int64_t gq = g - L.nr;
            const PairView P = pair_view(L, p);
            const PairGeom &G = L.geom[p];
            const int64_t i = gq - P.q_off;
            const double x1 = P.xy1[2 * i], y1 = P.xy1[2 * i + 1];
            QueryRec r;
            r.flags = 0;
            r.pair = p;
            r.pad[0] = r.pad[1] = 0;
            if (gq % kStabQB == 0) L.blkpair[gq / kStabQB] = p;
            r.A = r.B = r.C = r.key = r.aux0 = r.aux1 = r.E0 = r.E1 = 0.0f;
            if (!(finite64(x1) && finite64(y1))) set_status(L.status, kStNan);
            const double *F = P.F;
            // the line with FMAs: within a few ulps of its terms of the exact line
            const double a = fma(F[0], x1, fma(F[1], y1, F[2]));
            const double b = fma(F[3], x1, fma(F[4], y1, F[5]));
            const double c = fma(F[6], x1, fma(F[7], y1, F[8]));
            const float x1f = fabsf(d2f(x1)), y1f = fabsf(d2f(y1));
            const float ta = fabsf(G.Ff[0]) * x1f + fabsf(G.Ff[1]) * y1f + fabsf(G.Ff[2]);
            const float tb = fabsf(G.Ff[3]) * x1f + fabsf(G.Ff[4]) * y1f + fabsf(G.Ff[5]);
            const float tc = fabsf(G.Ff[6]) * x1f + fabsf(G.Ff[7]) * y1f + fabsf(G.Ff[8]);
            const float af = d2f(a), bf = d2f(b);
            const float N = sqrtf(af * af + bf * bf);
            const bool usable = isfinite(N) && finite64(c) && N > 1e-6f * (ta + tb) && N > 1e-30f;
            if (!usable) {
                // tiny or overflowing line: decide degeneracy exactly as the
                // brute force (a^2 + b^2 == 0 in its evaluation order)
                double ea, eb, ec;
                exact_line(P.F, x1, y1, ea, eb, ec);
                if (exact_norm(ea, eb) == 0.0) r.flags = EGM_FLAG_DEGENERATE_LINE;
                else r.flags = kQExactOnly;
            } else {
                const float invN = 1.0f / N;
                const double Cn = fma(a, G.cx, fma(b, G.cy, c));
                float A = af * invN, B = bf * invN, C = d2f(Cn) * invN;
                // the oracle's line differs from (a, b, c) by at most ~2 ulps of the terms
                const float da = 8.9e-16f * ta, db = 8.9e-16f * tb, dc = 8.9e-16f * tc;
                r.E0 = (da * G.cxf + db * G.cyf + dc) * invN * 1.001f;
                r.E1 = (da + db) * invN * 1.001f;
                if (G.mode == kModeAngular) {
                    // distance of the computed epipole from the line, bounded
                    // above: the exact line there is p . v (|v_k| <= vb_k), and
                    // the brute force's line is within a few ulps of its terms
                    // of the exact one
                    const float xe = fabsf(G.xef), ye = fabsf(G.yef);
                    const float rerr = 2.0e-15f * (ta * xe + tb * ye + tc);
                    const float rv = G.vb[0] * x1f + G.vb[1] * y1f + G.vb[2];
                    r.aux0 = (rv + rerr) * invN * 1.00001f + 1e-12f;
                    // line direction (B, -A) in the frame of u, reduced mod pi
                    r.key = fold_atan2(B * G.ux - A * G.uy, -(G.ux * A + G.uy * B));
                } else {
                    float cphi = -A * G.uy + B * G.ux;
                    if (cphi < 0.0f) { A = -A; B = -B; C = -C; cphi = -cphi; }
                    const float sphi = fabsf(A * G.ux + B * G.uy);
                    r.aux0 = cphi * (1.0f - 1e-6f);
                    r.aux1 = sphi * (1.0f + 1e-6f) + 1e-12f;
                    r.key = cphi > 0.5f ? -C / cphi : 0.0f;
                }
                r.A = A;
                r.B = B;
                r.C = C;
                if (!isfinite(r.C) || !isfinite(r.key)) r.flags = kQExactOnly;
            }
            L.qrec[gq] = r;
            if (L.qbkt) L.qbkt[gq] = (uint16_t)query_bucket(G, r);
            if (r.flags == 0u) {
                qgroup = (uint32_t)p;
                qa0 = __float_as_uint(r.aux0);
                qa1 = __float_as_uint(r.aux1);
                qk = __float_as_uint(fabsf(r.key));
            }
        }
        // warp-aggregated query extremes of each pair (the single-pair
        // stabbing kernel's per-level windows cover every query with them)
        if (__any_sync(0xffffffffu, qgroup != 0xffffffffu)) {
            const uint32_t qpeers = __match_any_sync(0xffffffffu, qgroup);
            const uint32_t a0x = __reduce_max_sync(qpeers, qa0);
            const uint32_t a0n = __reduce_min_sync(qpeers, qgroup == 0xffffffffu ? 0x7f800000u : qa0);
            const uint32_t a1x = __reduce_max_sync(qpeers, qa1);
            const uint32_t kx = __reduce_max_sync(qpeers, qk);
            if (qgroup != 0xffffffffu && lane == __ffs(qpeers) - 1) {
                PairGeom &G = L.geom[qgroup];
                atomicMax(&G.qa0max, a0x);
                atomicMin(&G.qa0min, a0n);
                atomicMax(&G.qa1max, a1x);
                atomicMax(&G.qkabs, kx);
            }
        }
        // warp-aggregated level statistics
        if (__any_sync(0xffffffffu, group != 0xffffffffu)) {
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
    // The last block to finish derives every pair's level layout (first sorted
    // position, bucket bits, table offset) from the final level counts.  A
    // single pair's layout is derived by the bucket-count kernel instead
    // (each of its blocks from the counts), which keeps this step -- a fence
    // and an atomic round trip -- off the single-pair chain.
    if (one || part == 2) return;
    // the block's writes are ordered before thread 0's fence by the barrier
    // (fences are cumulative), so one thread fences and counts the block
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(L.prep_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int p = threadIdx.x >> 5; p < L.npairs; p += blockDim.x >> 5) {
            PairGeom &G = L.geom[p];
            level_layout_lane(__ldcg(&G.cnt[lane]), G.start, G.bits, G.tab, kMaxBucketBits, lane);
        }
        if (threadIdx.x == 0) *L.prep_done = 0u;  // ready for the next launch
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
    return launch_pdl(geometry_kernel, dim3(L.npairs), dim3(32), 0, s, L);
}

cudaError_t launch_prep(const Launch &L, cudaStream_t s, int part) {
    const int64_t total = part == 1 ? L.nr : part == 2 ? L.nq : L.nr + L.nq;
    if (total == 0 && part != 1) return cudaSuccess;
    // one pair: blocks of 128 rows spread a pair's rows over more SMs (each
    // row is one pass of a latency-bound chain); a batch: blocks of 256 in
    // two resident waves
    const int T = L.npairs == 1 ? 128 : 256;
    int64_t blocks = (total + T - 1) / T;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;  // part 1 of a call without references: the tables and the layout
    return launch_pdl(prep_kernel, dim3((unsigned)blocks), dim3(T), 0, s, L, part);
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
