// adjoint.cu -- gradients of the navigator step (not in the paper: the
// differentiable use of the step).
//
// For a track whose step s ends on the surface F(x; theta) = 0 of the winning
// solid (F > 0 outside the solid), with local point x* = x + s u, local
// gradient g = grad_x F(x*) and den = g . u, the implicit-function rule gives
//     ds/dp = -R g / den,  ds/dd = -s R g / den,  ds/dt = +R g / den,
//     ds/dtheta = -(dF/dtheta)(x*) / den
// (R the solid's rotation, t its translation, theta its shape parameters; the
// mother has R = 1 and no translation).  The surface is the one the FP64
// routine of the forward step crossed (same arithmetic, so the same step).
// Where the surface is undefined (start inside a daughter, outside the mother,
// invalid input) or den = 0, the gradients are 0; a hit index >= nd (not one
// the forward step of this volume writes) also gives 0 and sets ST_BAD_INDEX
// in the volume's device status word.
//
// Geometry gradients are sums over tracks; they are reduced deterministically.
// Every block owns a fixed set of tiles of 256 tracks, ordered within the
// tile by their hit (a stable sort).  Within a tile each warp groups its
// lanes by owner (the winning daughter, or the mother's parameters) and sums
// every group in lane order; the warps then add their group sums into the
// block's shared accumulators one warp after the other (a warp's groups have
// distinct owners).  Block partials go to a
// caller-provided workspace and a second kernel adds them in block order.  No
// step depends on timing, so repeated calls give the same bits.
#include <cuda_runtime.h>

#include "geo_internal.h"
#include "launch.cuh"
#include "nav_common.cuh"
#include "shapes64.cuh"

namespace geonav {

constexpr int kAdjTile = 256;
constexpr int kGeo = 8;   // per owner: 3 translation + 5 shape-parameter components

// g = grad F at local x* on surface `face` of solid r, and dF/dtheta[5].
// (Every element is written by a select, so the arrays stay in registers.)
__device__ __forceinline__ void surface_grad64(const ShapeRec64& r, int face, const double* xs, double* g,
                                               double* dF) {
    const double* p = r.p;
    if (r.kind == KBOX) {
        const int ax = face >> 1;
        const double sg = (face & 1) ? 1.0 : -1.0;   // F = sg x_ax - h_ax
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            g[k] = ax == k ? sg : 0.0;
            dF[k] = ax == k ? -1.0 : 0.0;
        }
        dF[3] = dF[4] = 0.0;
        return;
    }
    if (face == 8 || face == 9) {                    // segments: F = -n.(x, y)
        const double* d = r.d;
        const double nx = face == 8 ? d[5] : d[7], ny = face == 8 ? d[6] : d[8];
        g[0] = -nx;
        g[1] = -ny;
        g[2] = 0.0;
        // d/dsphi of the face at sphi: e1.(x, y); of the face at sphi + dphi:
        // -e2.(x, y), for sphi and dphi alike; (sphi, dphi) are the parameter
        // slots 3, 4 of a tube segment and 0, 1 of a polycone
        const double de = face == 8 ? ny * xs[0] - nx * xs[1] : -(-ny * xs[0] + nx * xs[1]);
        const int is = r.kind == KPCON ? 0 : 3;
#pragma unroll
        for (int k = 0; k < 5; ++k) dF[k] = k == is ? de : (k == is + 1 && face == 9 ? de : 0.0);
        return;
    }
    if (r.kind == KPCON) {
        // end planes F = z[0] - z, z - z[nz-1]; section k: F = +-(rho^2 -
        // R(z)^2); the plane table gets no gradient
        dF[0] = dF[1] = dF[2] = dF[3] = dF[4] = 0.0;
        g[0] = g[1] = g[2] = 0.0;
        if (face == 4 || face == 5) {
            g[2] = face == 5 ? 1.0 : -1.0;
            return;
        }
        if (face < 16) return;
        const double* T = pcon_table(r.d);
        const int n = int(r.d[1]), k = (face - 16) >> 1;
        const bool outer = ((face - 16) & 1) == 0;
        const double* rr = T + (outer ? 2 * n : n);
        const double b = T[3 * n + (outer ? n - 1 : 0) + k];
        const double R = rr[k] + b * (xs[2] - T[k]);
        const double sg = outer ? 1.0 : -1.0;
        g[0] = sg * 2.0 * xs[0];
        g[1] = sg * 2.0 * xs[1];
        g[2] = -sg * 2.0 * R * b;
        return;
    }
    const bool tube = r.kind == KTUBE || r.kind == KTUBS;
    const double dz = tube ? p[2] : p[0];
    if (face == 4 || face == 5) {                    // F = +-z - dz
        g[0] = g[1] = 0.0;
        g[2] = face == 5 ? 1.0 : -1.0;
        dF[0] = tube ? 0.0 : -1.0;
        dF[1] = 0.0;
        dF[2] = tube ? -1.0 : 0.0;
        dF[3] = dF[4] = 0.0;
        return;
    }
    const bool outer = face == 6;
    const double sg = outer ? 1.0 : -1.0;            // outer: rho^2 - R^2, inner: R^2 - rho^2
    g[0] = sg * 2.0 * xs[0];
    g[1] = sg * 2.0 * xs[1];
    if (tube) {
        g[2] = 0.0;
        dF[0] = outer ? 0.0 : -sg * 2.0 * p[0];
        dF[1] = outer ? -sg * 2.0 * p[1] : 0.0;
        dF[2] = dF[3] = dF[4] = 0.0;
        return;
    }
    const double r1 = outer ? p[2] : p[1], r2 = outer ? p[4] : p[3];
    const double w = (xs[2] + dz) / (2.0 * dz);      // weight of the radius at +dz
    const double R = r1 + (r2 - r1) * w;
    const double dRdz = (r2 - r1) / (2.0 * dz);
    const double a1 = -sg * 2.0 * R * (1.0 - w), a2 = -sg * 2.0 * R * w;
    g[2] = -sg * 2.0 * R * dRdz;
    dF[0] = -sg * 2.0 * R * (r2 - r1) * (-xs[2] / (2.0 * dz * dz));   // dR/d(dz) at fixed z
    dF[1] = outer ? 0.0 : a1;
    dF[2] = outer ? a1 : 0.0;
    dF[3] = outer ? 0.0 : a2;
    dF[4] = outer ? a2 : 0.0;
}

constexpr int kAdjWarps = kAdjTile / 32;
constexpr int kTval = kAdjTile + 1;   // odd row length: the 8 components of one entry fall in different banks

__global__ void __launch_bounds__(kAdjTile) k_adjoint(VolView v, Basket b, const int32_t* __restrict__ hit,
                                                     const double* __restrict__ gstep, double* __restrict__ gp,
                                                     double* __restrict__ gd, double* __restrict__ partials) {
    extern __shared__ __align__(16) double smem_adj[];
    const int nown = v.nd + 1;                       // daughters, then the mother
    double* acc = smem_adj;                          // [nown * kGeo]
    double* gsum = acc + size_t(nown) * kGeo;        // [kAdjWarps][32][kGeo] group sums
    double* tval = gsum + kAdjWarps * 32 * kGeo;     // [kGeo][kTval] per-track contributions
    int* gown = reinterpret_cast<int*>(tval + kGeo * kTval);   // [kAdjWarps][32] group owners
    int* town = gown + kAdjWarps * 32;                // [kAdjTile] per-track owners
    int* skey = town + kAdjTile;                      // [kAdjTile] sort keys
    int* sidx = skey + kAdjTile;                      // [kAdjTile] the tile's track order
    int* wzero = sidx + kAdjTile;                     // [kAdjWarps] zeros of one radix pass
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nbits = 32 - __clz(v.nd + 2);           // keys 0 .. nd + 2
    for (int q = t; q < nown * kGeo; q += kAdjTile) acc[q] = 0.0;
    __syncthreads();
    const int64_t ntiles = (b.n + kAdjTile - 1) / kAdjTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // The tile's tracks ordered by their hit (a stable LSD radix sort,
        // one ballot per bit): the lanes of a warp then mostly run one
        // solid's FP64 routine, and a warp's owner groups are few.  Key 0:
        // no surface (outside, inside a daughter, past the basket's end), 1
        // the mother, j + 2 daughter j, nd + 2 a hit index out of range.
        int key = 0, idx = t;
        {
            const int64_t i0 = tile * kAdjTile + t;
            if (i0 < b.n) {
                const int h = hit[i0];
                key = h < -1 ? 0 : (h >= v.nd ? v.nd + 2 : h + 2);
            }
        }
        for (int bit = 0; bit < nbits; ++bit) {
            const bool one = (key >> bit) & 1;
            const unsigned ones = __ballot_sync(0xffffffffu, one);
            if (lane == 0) wzero[warp] = 32 - __popc(ones);
            __syncthreads();
            int before = 0, total = 0;   // zeros in the warps before this one, in the tile
            for (int w = 0; w < kAdjWarps; ++w) {
                const int z = wzero[w];
                total += z;
                if (w < warp) before += z;
            }
            const unsigned below = (1u << lane) - 1u;
            const int pos = one ? total + (warp * 32 - before) + __popc(ones & below)
                                : before + __popc(~ones & below);
            skey[pos] = key;
            sidx[pos] = idx;
            __syncthreads();
            key = skey[t];
            idx = sidx[t];
            __syncthreads();
        }
        const int64_t i = tile * kAdjTile + idx;
        int o = -1;
        double c[kGeo] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (i < b.n) {
            const double px = b.x[i], py = b.y[i], pz = b.z[i];
            const double qx = b.dx[i], qy = b.dy[i], qz = b.dz[i];
            const int h = hit[i];
            const double ws = gstep[i];
            double op[3] = {0, 0, 0}, od[3] = {0, 0, 0};
            if (h >= v.nd) atomicOr(v.status, ST_BAD_INDEX);   // not a hit of this volume: gradients 0
            if (h >= -1 && h < v.nd && valid_track(px, py, pz, qx, qy, qz)) {
                double x[3], u[3];
                int face = -1;
                double s;
                const ShapeRec64* r;
                if (h < 0) {
                    r = &v.m64;
                    x[0] = px; x[1] = py; x[2] = pz;
                    u[0] = qx; u[1] = qy; u[2] = qz;
                    s = dist_in64<true>(*r, x, u, &face);
                } else {
                    r = &v.d64[h];
                    to_local64(*r, px, py, pz, qx, qy, qz, x, u);
                    s = dist_out64<true>(*r, x, u, &face);
                }
                if (face >= 0 && isfinite(s)) {
                    const double xs[3] = {FMA(s, u[0], x[0]), FMA(s, u[1], x[1]), FMA(s, u[2], x[2])};
                    double g[3], dF[5];
                    surface_grad64(*r, face, xs, g, dF);
                    const double den = g[0] * u[0] + g[1] * u[1] + g[2] * u[2];
                    if (den != 0.0) {
                        double Rg[3];
                        if (h < 0) {
                            Rg[0] = g[0]; Rg[1] = g[1]; Rg[2] = g[2];
                        } else {
                            for (int k = 0; k < 3; ++k)
                                Rg[k] = r->R[3 * k] * g[0] + r->R[3 * k + 1] * g[1] + r->R[3 * k + 2] * g[2];
                        }
                        const double f = ws / den;
                        for (int k = 0; k < 3; ++k) {
                            op[k] = -f * Rg[k];
                            od[k] = -f * s * Rg[k];
                            if (h >= 0) c[k] = f * Rg[k];
                        }
                        for (int k = 0; k < 5; ++k) c[3 + k] = -f * dF[k];
                        o = h < 0 ? v.nd : h;
                    }
                }
            }
            for (int k = 0; k < 3; ++k) {
                gp[k * b.n + i] = op[k];
                gd[k * b.n + i] = od[k];
            }
        }
        // group the warp's lanes by owner (in order of first appearance); then
        // lane l sums component l % 8 of group l / 8 (and of group l / 8 + 4,
        // ... when there are more than four) over the warp's 32 entries in
        // lane order.  One FP64 add per entry serves four groups at once.
        double* wv = tval + warp * 32;                 // tval[k * kTval + warp * 32 + e]
        int* wo = town + warp * 32;
        wo[lane] = o;
#pragma unroll
        for (int k = 0; k < kGeo; ++k) wv[k * kTval + lane] = c[k];
        int ngroups = 0, myq = -1;
        unsigned pending = __ballot_sync(0xffffffffu, o >= 0);
        while (pending) {
            const int leader = __ffs(pending) - 1;
            const int q = __shfl_sync(0xffffffffu, o, leader);
            if (lane == ngroups) myq = q;
            ++ngroups;
            pending &= ~__ballot_sync(0xffffffffu, o == q);
        }
        __syncwarp();
        for (int base = 0; base < ngroups; base += 4) {
            const int g = base + (lane >> 3), k = lane & 7;
            const int q = __shfl_sync(0xffffffffu, myq, g & 31);
            double sum = 0.0;
            for (int e = 0; e < 32; ++e) sum += wo[e] == q ? wv[k * kTval + e] : 0.0;
            if (g < ngroups) {
                gsum[(warp * 32 + g) * kGeo + k] = sum;
                if (k == 0) gown[warp * 32 + g] = q;
            }
        }
        // the warps add their groups one after the other (fixed order); the
        // groups of one warp have distinct owners
        for (int w = 0; w < kAdjWarps; ++w) {
            __syncthreads();
            if (warp == w && lane < ngroups) {
                const int q = gown[w * 32 + lane];
#pragma unroll
                for (int k = 0; k < kGeo; ++k) acc[q * kGeo + k] += gsum[(w * 32 + lane) * kGeo + k];
            }
        }
        __syncthreads();
    }
    for (int q = t; q < nown * kGeo; q += kAdjTile) partials[size_t(blockIdx.x) * nown * kGeo + q] = acc[q];
}

// Sum of the block partials: one block per (owner, component) column; thread
// t adds the partials t, t + 256, ... in order, then a fixed shared-memory
// tree adds the 256 thread sums.  The order depends only on the block count.
__global__ void __launch_bounds__(256) k_adjoint_reduce(int nblocks, int nd, const double* __restrict__ partials,
                                                        double* __restrict__ gtrans, double* __restrict__ gparams) {
    __shared__ double red[256];
    const int nown = nd + 1;
    const int q = blockIdx.x;                        // column: owner q / kGeo, component q % kGeo
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) s += partials[size_t(b) * nown * kGeo + q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    s = red[0];
    const int o = q / kGeo, k = q % kGeo;
    if (k < 3) {
        if (o < nd && gtrans) gtrans[3 * o + k] = s;
    } else if (gparams) {
        gparams[5 * o + (k - 3)] = s;
    }
}

size_t adjoint_smem_bytes(int nd) {
    return (size_t(nd + 1) * kGeo + size_t(kAdjWarps) * 32 * kGeo + size_t(kGeo) * kTval) * sizeof(double) +
           (size_t(kAdjWarps) * 32 + 3 * size_t(kAdjTile) + kAdjWarps) * sizeof(int);
}

int adjoint_blocks(int64_t n, int num_sms) {
    const int64_t need = (n + kAdjTile - 1) / kAdjTile;
    const int64_t cap = int64_t(2) * num_sms;   // two resident blocks per SM (96 registers a thread)
    return int(need < 1 ? 1 : (need < cap ? need : cap));
}

size_t adjoint_workspace_bytes(int nd, int64_t n, int num_sms) {
    return size_t(adjoint_blocks(n, num_sms)) * size_t(nd + 1) * kGeo * sizeof(double);
}

cudaError_t launch_adjoint(const VolView& v, const Basket& b, const int32_t* hit, const double* gstep, double* gp,
                           double* gd, double* gtrans, double* gparams, double* workspace, cudaStream_t s,
                           int num_sms) {
    const int nb = adjoint_blocks(b.n, num_sms);
    const int smem = int(adjoint_smem_bytes(v.nd));
    cudaError_t e = prep(k_adjoint, smem);
    if (e != cudaSuccess) return e;
    k_adjoint<<<nb, kAdjTile, smem, s>>>(v, b, hit, gstep, gp, gd, workspace);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (gtrans || gparams) {
        k_adjoint_reduce<<<(v.nd + 1) * kGeo, 256, 0, s>>>(nb, v.nd, workspace, gtrans, gparams);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace geonav
