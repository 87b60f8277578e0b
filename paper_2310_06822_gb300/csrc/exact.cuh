// Exact sphere predicates on grid integers, shared by the labeler and the cascade.
//
// Values are integer multiples of 2^-qexp converted to int32 grid units and must
// satisfy |v| < 2^29, which bounds every intermediate: differences < 2^30, squared sums
// < 2^62 (int64), and the ray / plane / moving-point products < 2^126 (unsigned 128-bit).
#pragma once

#include "common.cuh"

namespace nbexact {

struct SphI {
    int c[3];
    int r;
    int v[3];
    int pad;
};

constexpr float kGridLimit = 536870912.0f;  // 2^29

__device__ __forceinline__ bool to_grid(float x, float scale, int &out) {
    float s = x * scale;  // scaling by a power of two is exact
    if (!(fabsf(s) < kGridLimit)) return false;  // also rejects NaN and inf
    int k = __float2int_rn(s);
    if ((float)k != s) return false;
    out = k;
    return true;
}

__device__ __forceinline__ long long sq(int a) { return (long long)a * (long long)a; }

template <int KIND>
__device__ __forceinline__ int union_hit(const int *Q, const SphI *sph, int ns, int qexp) {
    if constexpr (KIND == NB_POINT2) {
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            long long d2 = sq(Q[0] - S.c[0]) + sq(Q[1] - S.c[1]);
            if (d2 <= sq(S.r)) return 1;
        }
    } else if constexpr (KIND == NB_POINT3) {
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            long long d2 = sq(Q[0] - S.c[0]) + sq(Q[1] - S.c[1]) + sq(Q[2] - S.c[2]);
            if (d2 <= sq(S.r)) return 1;
        }
    } else if constexpr (KIND == NB_POINT4T) {
        // centre at time t is c + v t; scaled by 2^qexp every term is an integer:
        // d = (x - c) 2^qexp - v t  (units 2^-2qexp), test |d|^2 <= (r 2^qexp)^2
        const long long T = Q[3];
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            unsigned __int128 d2 = 0;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                long long d = (long long)(Q[i] - S.c[i]) * (1LL << qexp) - (long long)S.v[i] * T;
                unsigned long long a = d < 0 ? (unsigned long long)(-d) : (unsigned long long)d;
                d2 += (unsigned __int128)a * a;
            }
            unsigned long long rs = (unsigned long long)S.r << qexp;
            if (d2 <= (unsigned __int128)rs * rs) return 1;
        }
    } else if constexpr (KIND == NB_RAY3) {
        // half-line o + s d, s >= 0; w = c - o.  Closest point is o when w.d <= 0,
        // otherwise the foot of the perpendicular: |w|^2 |d|^2 - (w.d)^2 <= r^2 |d|^2,
        // rearranged as (|w|^2 - r^2) |d|^2 <= (w.d)^2 once |w|^2 > r^2.
        const long long DD = sq(Q[3]) + sq(Q[4]) + sq(Q[5]);
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            int w0 = S.c[0] - Q[0], w1 = S.c[1] - Q[1], w2 = S.c[2] - Q[2];
            long long WW = sq(w0) + sq(w1) + sq(w2);
            long long RR = sq(S.r);
            if (WW <= RR) return 1;
            long long SD = (long long)w0 * Q[3] + (long long)w1 * Q[4] + (long long)w2 * Q[5];
            if (SD <= 0) continue;
            unsigned __int128 lhs = (unsigned __int128)(unsigned long long)(WW - RR) * (unsigned long long)DD;
            unsigned __int128 rhs = (unsigned __int128)(unsigned long long)SD * (unsigned long long)SD;
            if (lhs <= rhs) return 1;
        }
    } else if constexpr (KIND == NB_PLANE3) {
        // plane {x : n.x = off}: (n.c - off)^2 <= r^2 |n|^2 (units 2^-4qexp)
        const long long NN = sq(Q[0]) + sq(Q[1]) + sq(Q[2]);
        const long long OFF = (long long)Q[3] * (1LL << qexp);
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            long long d = (long long)Q[0] * S.c[0] + (long long)Q[1] * S.c[1] + (long long)Q[2] * S.c[2] - OFF;
            unsigned long long a = d < 0 ? (unsigned long long)(-d) : (unsigned long long)d;
            if ((unsigned __int128)a * a <= (unsigned __int128)(unsigned long long)sq(S.r) * (unsigned long long)NN)
                return 1;
        }
    } else if constexpr (KIND == NB_BOX3) {
        // closed box: squared distance from the centre c to the box <= r^2
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            long long d2 = 0;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                int a = abs(S.c[i] - Q[i]) - Q[3 + i];
                if (a > 0) d2 += sq(a);
            }
            if (d2 <= sq(S.r)) return 1;
        }
    }
    return 0;
}

// ------------------------------------------------------------ FP32 pre-filter
// Most sphere tests are far from tangency.  The filter evaluates each predicate's
// quantities in FP32 from the exact float inputs (grid values are exact floats), with
// explicit round-to-nearest operations so that no contraction changes the count of
// roundings, and takes the decision only where the two sides differ by more than
// KAPPA = 2^-16 of the scale they are computed at; otherwise (|difference| within that)
// the exact integer test decides.  Every quantity below is a sum of at most a dozen
// rounded terms whose error is at most k u times that scale with k < 40, u = 2^-24
// (k u < 2.4e-6 < KAPPA / 6), and the threshold products add one more rounding each, so
// a filtered decision is always the exact predicate's.  Per quantity:
//   w = c - o (or x - c, c - b): relative error <= u per component;
//   |w|^2 = sum of fl(w_i^2): within gamma_5 |w|^2;  r^2 = fl(r r): within u r^2;
//   s = w . d (d exact): within gamma_5 sum |w_i d_i| <= gamma_5 |w| |d|;
//   |w x d|^2 from fl(fl(w_y d_z) - fl(w_z d_y)) components: within ~12 u |w|^2 |d|^2;
//   r^2 |d|^2: within gamma_3 r^2 |d|^2;
//   box a_i = |c_i - b_i| - e_i: d2 = sum max(a_i, 0)^2 within ~8 u sum (c_i - b_i)^2;
//   plane n . c - off: within gamma_4 (sum |n_i c_i| + |off|) =: gamma_4 M.
struct SphF {
    float c[3];
    float rr;  // fl(r r)
};

constexpr float KAPPA = 1.52587890625e-05f;  // 2^-16
constexpr float KLO = 1.0f - KAPPA, KHI = 1.0f + KAPPA;

// 1: certainly inside (or touching), 0: certainly outside, -1: undecided
__device__ __forceinline__ int cmp_filtered(float lhs, float rhs, float scale) {
    // decide lhs <= rhs when they differ by more than KAPPA * scale
    const float d = __fsub_rn(lhs, rhs), m = __fmul_rn(KAPPA, scale);
    if (d < -m) return 1;
    if (d > m) return 0;
    return -1;
}

template <int KIND>
__device__ __forceinline__ int union_hit_filtered(const float *qf, const int *Q, const SphF *sf, const SphI *sph,
                                                  int ns, int qexp) {
    if constexpr (KIND == NB_POINT2 || KIND == NB_POINT3) {
        constexpr int D = KIND == NB_POINT2 ? 2 : 3;
        for (int s = 0; s < ns; s++) {
            const SphF S = sf[s];
            float ww = 0.f;
#pragma unroll
            for (int i = 0; i < D; i++) {
                const float w = __fsub_rn(qf[i], S.c[i]);
                ww = __fadd_rn(ww, __fmul_rn(w, w));
            }
            const int f = cmp_filtered(ww, S.rr, __fadd_rn(ww, S.rr));
            if (f == 1) return 1;
            if (f == -1 && union_hit<KIND>(Q, sph + s, 1, qexp)) return 1;
        }
    } else if constexpr (KIND == NB_RAY3) {
        const float d0 = qf[3], d1 = qf[4], d2 = qf[5];
        const float dd = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
        for (int s = 0; s < ns; s++) {
            const SphF S = sf[s];
            const float w0 = __fsub_rn(S.c[0], qf[0]), w1 = __fsub_rn(S.c[1], qf[1]), w2 = __fsub_rn(S.c[2], qf[2]);
            const float ww = __fadd_rn(__fadd_rn(__fmul_rn(w0, w0), __fmul_rn(w1, w1)), __fmul_rn(w2, w2));
            // origin inside the ball: a hit
            const int fin = cmp_filtered(ww, S.rr, __fadd_rn(ww, S.rr));
            if (fin == 1) return 1;
            if (fin == -1) {
                if (union_hit<KIND>(Q, sph + s, 1, qexp)) return 1;
                continue;
            }
            // origin outside.  The line misses the ball when |w x d|^2 > r^2 |d|^2 (Lagrange:
            // |w|^2 |d|^2 - s^2 = |w x d|^2, s = w . d), and then so does the half-line, whatever
            // the sign of s; where the line meets the ball, the half-line does iff s > 0.
            const float pw = __fmul_rn(ww, dd);
            const float cx = __fsub_rn(__fmul_rn(w1, d2), __fmul_rn(w2, d1));
            const float cy = __fsub_rn(__fmul_rn(w2, d0), __fmul_rn(w0, d2));
            const float cz = __fsub_rn(__fmul_rn(w0, d1), __fmul_rn(w1, d0));
            const float x = __fadd_rn(__fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy)), __fmul_rn(cz, cz));
            const int f = cmp_filtered(x, __fmul_rn(S.rr, dd), pw);
            if (f == 0) continue;
            if (f == 1) {
                // the sign of s, certain once s^2 exceeds KAPPA |w|^2 |d|^2
                const float sd = __fadd_rn(__fadd_rn(__fmul_rn(w0, d0), __fmul_rn(w1, d1)), __fmul_rn(w2, d2));
                if (__fmul_rn(sd, sd) > __fmul_rn(KAPPA, pw)) {
                    if (sd > 0.f) return 1;
                    continue;  // the half-line points away: its closest point is the origin
                }
            }
            if (union_hit<KIND>(Q, sph + s, 1, qexp)) return 1;
        }
    } else if constexpr (KIND == NB_BOX3) {
        for (int s = 0; s < ns; s++) {
            const SphF S = sf[s];
            float d2 = 0.f, t2 = 0.f;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const float t = __fsub_rn(S.c[i], qf[i]);
                const float a = __fsub_rn(fabsf(t), qf[3 + i]);
                if (a > 0.f) d2 = __fadd_rn(d2, __fmul_rn(a, a));
                t2 = __fadd_rn(t2, __fmul_rn(t, t));
            }
            const int f = cmp_filtered(d2, S.rr, __fadd_rn(t2, S.rr));
            if (f == 1) return 1;
            if (f == -1 && union_hit<KIND>(Q, sph + s, 1, qexp)) return 1;
        }
    } else if constexpr (KIND == NB_PLANE3) {
        const float n0 = qf[0], n1 = qf[1], n2 = qf[2], off = qf[3];
        const float nn = __fadd_rn(__fadd_rn(__fmul_rn(n0, n0), __fmul_rn(n1, n1)), __fmul_rn(n2, n2));
        for (int s = 0; s < ns; s++) {
            const SphF S = sf[s];
            const float p0 = __fmul_rn(n0, S.c[0]), p1 = __fmul_rn(n1, S.c[1]), p2 = __fmul_rn(n2, S.c[2]);
            const float dv = __fsub_rn(__fadd_rn(__fadd_rn(p0, p1), p2), off);
            const float M = __fadd_rn(__fadd_rn(__fadd_rn(fabsf(p0), fabsf(p1)), fabsf(p2)), fabsf(off));
            const float rn = __fmul_rn(S.rr, nn);
            const int f = cmp_filtered(__fmul_rn(dv, dv), rn, __fadd_rn(__fmul_rn(M, M), rn));
            if (f == 1) return 1;
            if (f == -1 && union_hit<KIND>(Q, sph + s, 1, qexp)) return 1;
        }
    } else {
        return union_hit<KIND>(Q, sph, ns, qexp);
    }
    return 0;
}

}  // namespace nbexact
