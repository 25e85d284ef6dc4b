// vor_cells_thread.cuh -- helpers of the one-thread-per-cell projector.
//
// The candidate table of a thread lives in shared memory with the thread
// index fastest (conflict-free 16-byte loads).  The four sides of X are
// always candidates 0..3, so "c < 4" identifies them.
#pragma once

#include <cfloat>
#include <cmath>

#include "vor_device.cuh"
#include "vor_internal.h"

namespace vor {

namespace t1 {

struct Counters {
    unsigned long long rays, vtests, evals, exact, annulus, reruns, deferred, cands, maxe, widen;
};

enum { OK = 0, DEFER = 1, FAIL = 2 };

// candidate c of this thread: cb[c * NT] = (nx, ny), the line 2 <n, v - p> = c
// with c = |n|^2 (a site) or 2 |n|^2 (a side of X, candidates 0..3)
template <int NT>
struct Table {
    float2 *cb;
    __device__ __forceinline__ float2 get(int c) const { return cb[c * NT]; }
    __device__ __forceinline__ void put(int c, float2 v) const { cb[c * NT] = v; }
    __device__ __forceinline__ void line(int c, int &nx, int &ny, i64 &cc) const {
        const float2 q = get(c);
        nx = __float2int_rn(q.x);
        ny = __float2int_rn(q.y);
        cc = line_c(nx, ny, c < 4);
    }
};

__device__ __forceinline__ float2 cand_of(int nx, int ny) { return make_float2((float)nx, (float)ny); }

// reciprocal, PTX rcp.approx (maximum error 1 ulp over the whole range); the
// argument here is at least 1, so flushing denormals changes nothing
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Float filter of a candidate for the direction (fx, fy) = theta rounded to
// float: bounds U >= K >= L of its key K = <n, theta> / c.  The computed key
// errs by at most about 8u (|nx||tx| + |ny||ty|) / c (u = 2^-24: theta
// rounded to float, the dot product, c = nx^2 + ny^2 rounded, the 1-ulp
// reciprocal, the product); the tolerance (|nx| + |ny|) / c * max(|tx|,|ty|)
// * 2^-19 is 32u times an upper bound of the same factor, a margin of 4x
// that also covers the rounding of the tolerance and of k +- tol.
__device__ __forceinline__ void filter_keys(float2 q, bool side, float fx, float fy, float eth,
                                            float &U, float &L) {
    const float cf = fmaf(q.x, q.x, q.y * q.y) * (side ? 2.f : 1.f);
    const float rc = rcp_approx(cf);
    const float den = fmaf(q.x, fx, q.y * fy);
    const float tol = (fabsf(q.x) + fabsf(q.y)) * rc * eth;
    U = fmaf(den, rc, tol);
    L = fmaf(den, rc, -tol);
}

// a strictly more counter-clockwise than b (normals in one open half-plane)
template <int NT>
__device__ __forceinline__ bool more_ccw(const Table<NT> &T, int a, int b) {
    int ax, ay, bx, by;
    i64 ca, cb;
    T.line(a, ax, ay, ca);
    T.line(b, bx, by, cb);
    return (i64)bx * ay - (i64)by * ax > 0;
}

// Exact endpoint over the candidates whose filter upper bound reaches thr
// (all candidates when use_thr is false); ties resolved per Remark A.4.
template <int NT>
__device__ void exact_argmax(const Table<NT> &T, int C, i64 tx, i64 ty, float fx, float fy,
                             float eth, bool use_thr, float thr, int &ccw, int &cw) {
    int best = -1;
    ccw = cw = -1;
    i128 bd = 0;
    i64 bc = 1;
    for (int c = 0; c < C; c++) {
        if (use_thr) {
            float U, L;
            filter_keys(T.get(c), c < 4, fx, fy, eth, U, L);
            if (!(U >= thr)) continue;
        }
        int nx, ny;
        i64 cc;
        T.line(c, nx, ny, cc);
        const i128 d = dot128(nx, ny, tx, ty);
        if (d <= 0) continue;
        if (best < 0) { best = c; ccw = cw = c; bd = d; bc = cc; continue; }
        const i128 lhs = d * (i128)bc, rhs = bd * (i128)cc;     // key(c) vs key(best)
        if (lhs > rhs) { best = c; ccw = cw = c; bd = d; bc = cc; }
        else if (lhs == rhs) {
            if (more_ccw(T, c, ccw)) ccw = c;
            if (more_ccw(T, cw, c)) cw = c;
        }
    }
}

__device__ __forceinline__ int cross_sign(i64 ax, i64 ay, i64 bx, i64 by) {
    const float p = (float)ax * (float)by, q = (float)ay * (float)bx;
    const float v = p - q, bound = (fabsf(p) + fabsf(q)) * 0x1p-20f;
    if (v > bound) return 1;
    if (v < -bound) return -1;
    const i128 e = cross128(ax, ay, bx, by);
    return e > 0 ? 1 : (e < 0 ? -1 : 0);
}

}  // namespace t1


}  // namespace vor
