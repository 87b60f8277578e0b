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

}  // namespace nbexact
