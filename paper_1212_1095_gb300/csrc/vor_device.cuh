// vor_device.cuh -- device-side building blocks of the projector kernels.
//
// Geometry, in coordinates relative to the cell's site p (the paper's
// Section 3-4 quantities written for integer sites):
//   a candidate line is { v : 2 <n, v> = c }:
//     neighbour site a:  n = a - p,            c = |n|^2   (bisector of p and a)
//     side of X:         n = (mirror - p) / 2, c = 2|n|^2  (the side itself; the
//                        bisector of p and its reflection across the side)
//   a ray p + t*theta meets the line at t = c / (2 <n, theta>) if <n, theta> > 0,
//   so the endpoint T(p, theta) of eq. (2.1) is the line with the largest
//   key K = <n, theta> / c (the smallest t).
// |n| < 2^20, c < 2^41 and every direction component stays below 2^62, so the
// exact predicates below fit in signed 128-bit integers.
#pragma once

#include <cstdint>

typedef long long i64;
typedef __int128 i128;

namespace vor {

// ---------------------------------------------------------------------------
// exact predicates
// ---------------------------------------------------------------------------

__device__ __forceinline__ i64 line_c(int nx, int ny, bool side) {
    i64 c = (i64)nx * nx + (i64)ny * ny;
    return side ? 2 * c : c;
}

__device__ __forceinline__ i128 dot128(int nx, int ny, i64 tx, i64 ty) {
    return (i128)nx * tx + (i128)ny * ty;
}

__device__ __forceinline__ i128 cross128(i64 ax, i64 ay, i64 bx, i64 by) {
    return (i128)ax * by - (i128)ay * bx;
}

// Half-plane of a direction for the counter-clockwise order starting at the
// positive x axis: 0 for angles in [0, pi), 1 for [pi, 2 pi).
__device__ __forceinline__ int half_of(int x, int y) { return (y > 0 || (y == 0 && x > 0)) ? 0 : 1; }

// Polar angle of (ax, ay) strictly below that of (bx, by), angles in [0, 2 pi).
__device__ __forceinline__ bool angle_less(int ax, int ay, int bx, int by) {
    int ha = half_of(ax, ay), hb = half_of(bx, by);
    if (ha != hb) return ha < hb;
    return (i64)ax * by - (i64)ay * bx > 0;
}

// Intersection u of two candidate lines: u - p = N / D with
//   N = (c1 n2y - c2 n1y, c2 n1x - c1 n2x),  D = 2 (n1x n2y - n1y n2x).
// |N| < 2^62 and |D| < 2^42.
__device__ __forceinline__ void intersect(int n1x, int n1y, i64 c1, int n2x, int n2y, i64 c2,
                                          i64 &Nx, i64 &Ny, i64 &D) {
    Nx = c1 * n2y - c2 * n1y;
    Ny = c2 * n1x - c1 * n2x;
    D = 2 * ((i64)n1x * n2y - (i64)n1y * n2x);
}

// ---------------------------------------------------------------------------
// group (G lanes of one warp working on one cell) helpers
// ---------------------------------------------------------------------------

template <int G>
__device__ __forceinline__ float group_max(float v, unsigned gmask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(gmask, v, off, G));
    return v;
}

template <int G>
__device__ __forceinline__ int group_sum(int v, unsigned gmask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(gmask, v, off, G);
    return v;
}

template <int G>
__device__ __forceinline__ int group_or(int v, unsigned gmask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v |= __shfl_xor_sync(gmask, v, off, G);
    return v;
}

template <int G>
__device__ __forceinline__ void group_sync(unsigned gmask) {
    if (G > 1) __syncwarp(gmask);
}

}  // namespace vor
