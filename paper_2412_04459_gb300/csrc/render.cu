// Forward and backward compositing of the sorted tile lists (sm_103a).
//
// One CTA per 16x16 tile, one thread per pixel; warp w covers the 8x4 pixel
// block (w & 1, w >> 1) of its tile.  The tile's list is staged through
// shared memory 256 entries at a time (one entry per thread: value, then the
// voxel's 64-byte record as four 16-byte loads); every pixel then walks the
// staged entries, skipping those whose sign bits differ from its own
// (Sec. B.1) and those its ray misses (ray-AABB, Sec. A.2).  The entry and
// exit planes of a voxel follow from the sign bits, so the slab test is six
// multiplies by 1/r_d and four min/max.
//
// Forward (Sec. 3.1.2, Eq. alpha_blend, Eq. supp_alpha_comp, Sec. A.4):
//   K samples per segment, trilinear raw density, explin, per-sample
//   e_k = exp(-(l/K) explin(v_k)); 1 - alpha = prod_k e_k; local depth
//   d = sum_k prod_{j<k} e_j (1 - e_k) t_k; C += T alpha c, D += T d,
//   T *= 1 - alpha; the warp's pixels stop after the voxel that leaves
//   T < t_stop and the CTA leaves the list once all its pixels stopped.
//
// Backward, back to front from the saved (T_final, last).  With x_i the
// optical depth of voxel i (T_{i+1} = T_i exp(-x_i)) and, accumulated from
// the back, SC_i = sum_{j>i} T_j alpha_j c_j + T_final bg and
// SD_i = sum_{j>i} T_j d_j:
//   dC/dx_i = T_{i+1} c_i - SC_i,  dA/dx_i = T_final,  dD/dx_i|_T = -SD_i,
//   dC/dc_i = T_i alpha_i,
//   dd_i/dx_ik = P_{k+1} t_k - sum_{m>k} P_m (1 - e_m) t_m  (P_k = prod_{j<k} e_j;
//                the general form of the K <= 3 closed forms of Sec. A.4),
//   dx_ik/dv_k = (l/K) explin'(v_k), dv_k/dV_c = trilinear weight of corner c.
// T_i is recovered as T_{i+1} / exp(-x_i).  Pixels whose T_final is below
// 1e-30 (where that division loses precision) take a front-to-back second
// phase instead, with SC_i, SD_i from totals recomputed in a first sweep.
// The per-voxel gradients (8 corner densities, 3 colour channels) of the
// lanes that hit the same entry are summed in the warp before the atomics.
#include "svr_internal.cuh"

namespace svr {

constexpr int kChunk = 256;

// Staged entry (96 bytes).  a/b hold the entry (near) and exit (far) planes
// relative to the ray origin for the entry's sign pattern; s rides in a.w.
struct Entry {
    float4 a;   // near.xyz, sign bits (int)
    float4 b;   // far.xyz, 1 / size
    float4 c;   // (lo - r_o) / size, voxel id (int)
    float4 g0;  // corner densities 0..3
    float4 g1;  // corner densities 4..7
    float4 col; // colour, clamp bits
};

__device__ __forceinline__ void stage_entry(Entry &e, uint32_t val, const Record *__restrict__ rec) {
    const uint32_t s = val >> 29;
    const uint32_t vid = val & 0x1FFFFFFFu;
    const Record *r = rec + vid;
    const float4 r0 = __ldg(&r->r0);
    const float lx = r0.x, ly = r0.y, lz = r0.z, size = r0.w;
    const float hx = lx + size, hy = ly + size, hz = lz + size;
    const float inv = 1.0f / size;
    e.a = make_float4((s & 4) ? hx : lx, (s & 2) ? hy : ly, (s & 1) ? hz : lz, __int_as_float((int)s));
    e.b = make_float4((s & 4) ? lx : hx, (s & 2) ? ly : hy, (s & 1) ? lz : hz, inv);
    e.c = make_float4(lx * inv, ly * inv, lz * inv, __int_as_float((int)vid));
    e.g0 = __ldg(&r->r1);
    e.g1 = __ldg(&r->r2);
    e.col = __ldg(&r->r3);
}

// Trilinear interpolation of Eq. interp; corner bits (x, y, z), x most significant.
__device__ __forceinline__ float trilerp(const float4 &g0, const float4 &g1, float qx, float qy, float qz) {
    const float c00 = fmaf(qz, g0.y - g0.x, g0.x);  // 000, 001
    const float c01 = fmaf(qz, g0.w - g0.z, g0.z);  // 010, 011
    const float c10 = fmaf(qz, g1.y - g1.x, g1.x);  // 100, 101
    const float c11 = fmaf(qz, g1.w - g1.z, g1.z);  // 110, 111
    const float c0 = fmaf(qy, c01 - c00, c00);
    const float c1 = fmaf(qy, c11 - c10, c10);
    return fmaf(qx, c1 - c0, c0);
}

struct PixelRay {
    float3 rd, inv;
    float rdn;
    int s;
    int x, y;
    bool inside;
};

__device__ __forceinline__ PixelRay pixel_ray(const DevCam &cam, int tile) {
    PixelRay p;
    const int tx = tile % cam.ntx, ty = tile / cam.ntx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    p.x = tx * 16 + (warp & 1) * 8 + (lane & 7);
    p.y = ty * 16 + (warp >> 1) * 4 + (lane >> 3);
    p.inside = p.x < cam.W && p.y < cam.H;
    p.rd = pixel_dir(cam, p.x, p.y);
    p.s = sign_bits(p.rd);
    // +0.0 for a zero component so that 1/r_d has the sign of the sign bits
    p.inv = make_float3(1.0f / (p.rd.x + 0.0f), 1.0f / (p.rd.y + 0.0f), 1.0f / (p.rd.z + 0.0f));
    p.rdn = sqrtf(p.rd.x * p.rd.x + p.rd.y * p.rd.y + p.rd.z * p.rd.z);
    return p;
}

// Slab test against a staged entry whose sign bits match the ray's.
__device__ __forceinline__ bool slab(const Entry &e, const PixelRay &p, float &a, float &b) {
    a = fmaxf(fmaxf(e.a.x * p.inv.x, e.a.y * p.inv.y), e.a.z * p.inv.z);
    b = fminf(fminf(e.b.x * p.inv.x, e.b.y * p.inv.y), e.b.z * p.inv.z);
    return a <= b && a > 0.f;
}

// ------------------------------------------------------------------ forward

// Local depth and transmittance factor of a hit (forward recompute).
template <int K>
__device__ __forceinline__ void hit_fwd(const Entry &e, const PixelRay &p, float a, float b, float &trans,
                                        float &dloc) {
    const float inv_k = 1.0f / K;
    const float seg = b - a;
    const float xs = seg * p.rdn * inv_k;
    const float step = seg * inv_k;
    const float inv_size = e.b.w;
    const float rx = p.rd.x * inv_size, ry = p.rd.y * inv_size, rz = p.rd.z * inv_size;
    float t = fmaf(0.5f, step, a);
    float P = 1.f, d = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float v = trilerp(e.g0, e.g1, fmaf(t, rx, -e.c.x), fmaf(t, ry, -e.c.y), fmaf(t, rz, -e.c.z));
        const float ek = __expf(-xs * explin(v));
        d = fmaf(P * (1.f - ek), t, d);
        P *= ek;
        t += step;
    }
    trans = P;
    dloc = d;
}


// STATS: also count, per pixel, the list entries with its sign bits that it
// examined and the hits it composited (int2 per pixel), for work accounting.
template <int K, bool STATS>
__global__ void __launch_bounds__(kChunk) k_render_fwd(FrameDev f, const uint32_t *__restrict__ vals,
                                                       float *__restrict__ out_rgb, float *__restrict__ out_depth,
                                                       float *__restrict__ out_alpha, float *__restrict__ out_T,
                                                       int32_t *__restrict__ out_last, int2 *__restrict__ stats) {
    __shared__ Entry ent[kChunk];
    const int tile = blockIdx.x;
    const PixelRay p = pixel_ray(f.cam, tile);
    const uint2 rg = f.ranges[tile];
    const int beg = (int)rg.x, end = (int)rg.y;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    int last = end - 1;
    bool done = !p.inside;
    int n_cand = 0, n_hit = 0;

    for (int base = beg; base < end; base += kChunk) {
        if (__syncthreads_count(!done) == 0) break;
        const int i = base + threadIdx.x;
        if (i < end) stage_entry(ent[threadIdx.x], vals[i], f.rec);
        __syncthreads();
        const int n = min(kChunk, end - base);
        if (!done) {
            for (int j = 0; j < n; ++j) {
                const Entry &e = ent[j];
                if (__float_as_int(e.a.w) != p.s) continue;
                if (STATS) ++n_cand;
                float a, b;
                if (!slab(e, p, a, b)) continue;
                if (STATS) ++n_hit;
                float P, dloc;
                hit_fwd<K>(e, p, a, b, P, dloc);
                const float w = T * (1.f - P);
                C0 = fmaf(w, e.col.x, C0);
                C1 = fmaf(w, e.col.y, C1);
                C2 = fmaf(w, e.col.z, C2);
                D = fmaf(T, dloc, D);
                T *= P;
                if (T < f.t_stop) {
                    done = true;
                    last = base + j;
                    break;
                }
            }
        }
    }
    if (p.inside) {
        const size_t HW = (size_t)f.cam.W * f.cam.H;
        const size_t o = (size_t)p.y * f.cam.W + p.x;
        out_rgb[o] = fmaf(T, f.bg[0], C0);
        out_rgb[HW + o] = fmaf(T, f.bg[1], C1);
        out_rgb[2 * HW + o] = fmaf(T, f.bg[2], C2);
        out_depth[o] = D;
        out_alpha[o] = 1.f - T;
        out_T[o] = T;
        out_last[o] = last;
        if (STATS) stats[o] = make_int2(n_cand, n_hit);
    }
}

// ----------------------------------------------------------------- backward

struct PixelGrad {
    float gC0, gC1, gC2, gD, gA;
    float Tfin;
};

// Gradient contributions of one hit.  T_i: transmittance in front of the
// voxel; T_after = T_i * prod_k e_k; SC, SD: sums behind it.  Adds the local
// quantities the caller needs to update its suffix or prefix sums.
template <int K>
__device__ __forceinline__ void hit_grad(const Entry &e, const PixelRay &p, const PixelGrad &g, float a, float b,
                                         float T_i, float T_after, const float SC[3], float SD, float dgeo[8],
                                         float dcol[3]) {
    const float inv_k = 1.0f / K;
    const float seg = b - a;
    const float xs = seg * p.rdn * inv_k;
    const float step = seg * inv_k;
    const float inv_size = e.b.w;
    const float rx = p.rd.x * inv_size, ry = p.rd.y * inv_size, rz = p.rd.z * inv_size;
    float tk[K], ek[K], qx[K], qy[K], qz[K], dsig[K];
    float t = fmaf(0.5f, step, a);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        qx[k] = fmaf(t, rx, -e.c.x);
        qy[k] = fmaf(t, ry, -e.c.y);
        qz[k] = fmaf(t, rz, -e.c.z);
        const float v = trilerp(e.g0, e.g1, qx[k], qy[k], qz[k]);
        const float sig = explin(v);
        dsig[k] = v > 1.1f ? 1.f : sig * 0.909090909f;
        ek[k] = __expf(-xs * sig);
        tk[k] = t;
        t += step;
    }
    float trans = 1.f;
#pragma unroll
    for (int k = 0; k < K; ++k) trans *= ek[k];
    const float alpha = 1.f - trans;
    const float w = T_i * alpha;
    dcol[0] = w * g.gC0;
    dcol[1] = w * g.gC1;
    dcol[2] = w * g.gC2;
    // dL/dx_i through C, A and the transmittance of later voxels in D
    const float gx = g.gC0 * fmaf(T_after, e.col.x, -SC[0]) + g.gC1 * fmaf(T_after, e.col.y, -SC[1]) +
                     g.gC2 * fmaf(T_after, e.col.z, -SC[2]) + g.gA * g.Tfin - g.gD * SD;
    // per-sample depth term, suffix Q_k = sum_{m>k} P_m (1 - e_m) t_m
    float Pk[K + 1];
    Pk[0] = 1.f;
#pragma unroll
    for (int k = 0; k < K; ++k) Pk[k + 1] = Pk[k] * ek[k];
    float Q = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) dgeo[c] = 0.f;
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
        const float gxk = fmaf(g.gD * T_i, fmaf(Pk[k + 1], tk[k], -Q), gx);
        const float dv = gxk * xs * dsig[k];
        const float ux = 1.f - qx[k], uy = 1.f - qy[k], uz = 1.f - qz[k];
        const float w00 = ux * uy, w01 = ux * qy[k], w10 = qx[k] * uy, w11 = qx[k] * qy[k];
        dgeo[0] = fmaf(dv, w00 * uz, dgeo[0]);
        dgeo[1] = fmaf(dv, w00 * qz[k], dgeo[1]);
        dgeo[2] = fmaf(dv, w01 * uz, dgeo[2]);
        dgeo[3] = fmaf(dv, w01 * qz[k], dgeo[3]);
        dgeo[4] = fmaf(dv, w10 * uz, dgeo[4]);
        dgeo[5] = fmaf(dv, w10 * qz[k], dgeo[5]);
        dgeo[6] = fmaf(dv, w11 * uz, dgeo[6]);
        dgeo[7] = fmaf(dv, w11 * qz[k], dgeo[7]);
        Q = fmaf(Pk[k] * (1.f - ek[k]), tk[k], Q);
    }
}

// Sum the 11 gradient values over the lanes that hit the entry and add them
// to the global accumulators.
__device__ __forceinline__ void flush_grad(bool hit, float dgeo[8], float dcol[3], const int32_t *__restrict__ cidx,
                                           int vid, float *__restrict__ d_grid, float *__restrict__ acc_col) {
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    if (__popc(m) == 1) {
        if (hit) {
#pragma unroll
            for (int c = 0; c < 8; ++c) atomicAdd(d_grid + __ldg(cidx + c), dgeo[c]);
            atomicAdd(acc_col + 3 * vid + 0, dcol[0]);
            atomicAdd(acc_col + 3 * vid + 1, dcol[1]);
            atomicAdd(acc_col + 3 * vid + 2, dcol[2]);
        }
        return;
    }
    if (!hit) {
#pragma unroll
        for (int c = 0; c < 8; ++c) dgeo[c] = 0.f;
        dcol[0] = dcol[1] = dcol[2] = 0.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < 8; ++c) dgeo[c] += __shfl_xor_sync(0xffffffffu, dgeo[c], o);
        dcol[0] += __shfl_xor_sync(0xffffffffu, dcol[0], o);
        dcol[1] += __shfl_xor_sync(0xffffffffu, dcol[1], o);
        dcol[2] += __shfl_xor_sync(0xffffffffu, dcol[2], o);
    }
    if (lane == __ffs(m) - 1) {
#pragma unroll
        for (int c = 0; c < 8; ++c) atomicAdd(d_grid + __ldg(cidx + c), dgeo[c]);
        atomicAdd(acc_col + 3 * vid + 0, dcol[0]);
        atomicAdd(acc_col + 3 * vid + 1, dcol[1]);
        atomicAdd(acc_col + 3 * vid + 2, dcol[2]);
    }
}

template <int K>
__global__ void __launch_bounds__(kChunk) k_render_bwd(FrameDev f, const uint32_t *__restrict__ vals,
                                                       const float *__restrict__ d_rgb,
                                                       const float *__restrict__ d_depth,
                                                       const float *__restrict__ d_alpha,
                                                       const float *__restrict__ in_T,
                                                       const int32_t *__restrict__ in_last,
                                                       float *__restrict__ d_grid) {
    __shared__ Entry ent[kChunk];
    __shared__ int max_last;
    const int tile = blockIdx.x;
    const PixelRay p = pixel_ray(f.cam, tile);
    const uint2 rg = f.ranges[tile];
    const int beg = (int)rg.x;
    const size_t HW = (size_t)f.cam.W * f.cam.H;
    const size_t o = (size_t)p.y * f.cam.W + p.x;

    PixelGrad g = {0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
    int last = beg - 1;
    if (p.inside) {
        if (d_rgb) {
            g.gC0 = d_rgb[o];
            g.gC1 = d_rgb[HW + o];
            g.gC2 = d_rgb[2 * HW + o];
        }
        if (d_depth) g.gD = d_depth[o];
        if (d_alpha) g.gA = d_alpha[o];
        g.Tfin = in_T[o];
        last = max(beg - 1, min(in_last[o], (int)rg.y - 1));   // stay inside the tile's list
    }
    const bool fallback = p.inside && last >= beg && g.Tfin < 1e-30f;
    const bool active = p.inside && last >= beg && !fallback;

    if (threadIdx.x == 0) max_last = beg - 1;
    __syncthreads();
    if (p.inside && last >= beg) atomicMax(&max_last, last);
    __syncthreads();
    const int hi_all = max_last + 1;

    // ---- back to front
    float T_after = g.Tfin;
    float SC[3] = {g.Tfin * f.bg[0], g.Tfin * f.bg[1], g.Tfin * f.bg[2]};
    float SD = 0.f;
    for (int hi = hi_all; hi > beg; hi -= kChunk) {
        const int lo = max(beg, hi - kChunk);
        __syncthreads();
        const int i = lo + threadIdx.x;
        if (i < hi) stage_entry(ent[threadIdx.x], vals[i], f.rec);
        __syncthreads();
        for (int j = hi - 1 - lo; j >= 0; --j) {
            const Entry &e = ent[j];
            float a = 0.f, b = 0.f;
            const bool hit = active && (lo + j) <= last && __float_as_int(e.a.w) == p.s && slab(e, p, a, b);
            float dgeo[8], dcol[3];
            if (hit) {
                float trans, dloc;
                hit_fwd<K>(e, p, a, b, trans, dloc);
                const float T_i = T_after / trans;
                hit_grad<K>(e, p, g, a, b, T_i, T_after, SC, SD, dgeo, dcol);
                const float w = T_i * (1.f - trans);
                SC[0] = fmaf(w, e.col.x, SC[0]);
                SC[1] = fmaf(w, e.col.y, SC[1]);
                SC[2] = fmaf(w, e.col.z, SC[2]);
                SD = fmaf(T_i, dloc, SD);
                T_after = T_i;
            }
            const int vid = __float_as_int(e.c.w);
            flush_grad(hit, dgeo, dcol, f.corner_idx + 8 * (size_t)vid, vid, d_grid, f.dcol);
        }
    }

    // ---- front to back for pixels whose T_final underflowed
    if (__syncthreads_or(fallback)) {
        // sweep 1: totals
        float T = 1.f, Ct[3] = {0.f, 0.f, 0.f}, Dt = 0.f;
        for (int lo = beg; lo < hi_all; lo += kChunk) {
            const int hi = min(hi_all, lo + kChunk);
            __syncthreads();
            const int i = lo + threadIdx.x;
            if (i < hi) stage_entry(ent[threadIdx.x], vals[i], f.rec);
            __syncthreads();
            if (fallback) {
                for (int j = 0; j < hi - lo && lo + j <= last; ++j) {
                    const Entry &e = ent[j];
                    float a, b;
                    if (__float_as_int(e.a.w) != p.s || !slab(e, p, a, b)) continue;
                    float trans, dloc;
                    hit_fwd<K>(e, p, a, b, trans, dloc);
                    const float w = T * (1.f - trans);
                    Ct[0] = fmaf(w, e.col.x, Ct[0]);
                    Ct[1] = fmaf(w, e.col.y, Ct[1]);
                    Ct[2] = fmaf(w, e.col.z, Ct[2]);
                    Dt = fmaf(T, dloc, Dt);
                    T *= trans;
                }
            }
        }
        Ct[0] = fmaf(T, f.bg[0], Ct[0]);
        Ct[1] = fmaf(T, f.bg[1], Ct[1]);
        Ct[2] = fmaf(T, f.bg[2], Ct[2]);
        // sweep 2: gradients with SC = total - prefix
        float Tf = 1.f, PC[3] = {0.f, 0.f, 0.f}, PD = 0.f;
        for (int lo = beg; lo < hi_all; lo += kChunk) {
            const int hi = min(hi_all, lo + kChunk);
            __syncthreads();
            const int i = lo + threadIdx.x;
            if (i < hi) stage_entry(ent[threadIdx.x], vals[i], f.rec);
            __syncthreads();
            for (int j = 0; j < hi - lo; ++j) {
                const Entry &e = ent[j];
                float a = 0.f, b = 0.f;
                const bool hit = fallback && (lo + j) <= last && __float_as_int(e.a.w) == p.s && slab(e, p, a, b);
                float dgeo[8], dcol[3];
                if (hit) {
                    float trans, dloc;
                    hit_fwd<K>(e, p, a, b, trans, dloc);
                    const float w = Tf * (1.f - trans);
                    PC[0] = fmaf(w, e.col.x, PC[0]);
                    PC[1] = fmaf(w, e.col.y, PC[1]);
                    PC[2] = fmaf(w, e.col.z, PC[2]);
                    PD = fmaf(Tf, dloc, PD);
                    const float SCi[3] = {Ct[0] - PC[0], Ct[1] - PC[1], Ct[2] - PC[2]};
                    const float Ta = Tf * trans;
                    hit_grad<K>(e, p, g, a, b, Tf, Ta, SCi, Dt - PD, dgeo, dcol);
                    Tf = Ta;
                }
                const int vid = __float_as_int(e.c.w);
                flush_grad(hit, dgeo, dcol, f.corner_idx + 8 * (size_t)vid, vid, d_grid, f.dcol);
            }
        }
    }
}

// Per voxel: dL/dsh[n][c] = Y_n(d) * dL/dc_c where the channel was > 0 before
// the clamp (Eq. vox_color), zero for voxels not in view.
__global__ void __launch_bounds__(256) k_voxel_bwd(FrameDev f, float *__restrict__ d_sh) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= f.n_vox) return;
    float4 *out = reinterpret_cast<float4 *>(d_sh + 48 * v);
    if (f.count[v] == 0) {
#pragma unroll
        for (int q = 0; q < 12; ++q) out[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const unsigned bits = __float_as_uint(f.rec[v].r3.w);
    const float g0 = (bits & 1u) ? f.dcol[3 * v + 0] : 0.f;
    const float g1 = (bits & 2u) ? f.dcol[3 * v + 1] : 0.f;
    const float g2 = (bits & 4u) ? f.dcol[3 * v + 2] : 0.f;
    float dx = f.centre[3 * v + 0] - f.cam.ro[0];
    float dy = f.centre[3 * v + 1] - f.cam.ro[1];
    float dz = f.centre[3 * v + 2] - f.cam.ro[2];
    const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    float Y[16];
    sh_basis(dx * inv, dy * inv, dz * inv, Y);
    float o[48];
#pragma unroll
    for (int n = 0; n < 16; ++n) {
        o[3 * n + 0] = Y[n] * g0;
        o[3 * n + 1] = Y[n] * g1;
        o[3 * n + 2] = Y[n] * g2;
    }
#pragma unroll
    for (int q = 0; q < 12; ++q) out[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_render_fwd(const FrameDev &f, int sorted_alt, float *rgb, float *depth, float *alpha,
                              float *T_final, int32_t *last, int2 *stats, cudaStream_t s) {
    const int ntiles = f.cam.ntx * f.cam.nty;
    const uint32_t *vals = f.vals[sorted_alt];
#define SVR_FWD(KK, ST) k_render_fwd<KK, ST><<<ntiles, kChunk, 0, s>>>(f, vals, rgb, depth, alpha, T_final, last, stats)
    if (stats) {
        switch (f.K) {
            case 1: SVR_FWD(1, true); break;
            case 2: SVR_FWD(2, true); break;
            case 3: SVR_FWD(3, true); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (f.K) {
            case 1: SVR_FWD(1, false); break;
            case 2: SVR_FWD(2, false); break;
            case 3: SVR_FWD(3, false); break;
            default: return cudaErrorInvalidValue;
        }
    }
#undef SVR_FWD
    return cudaGetLastError();
}

cudaError_t launch_render_bwd(const FrameDev &f, int sorted_alt, const float *d_rgb, const float *d_depth,
                              const float *d_alpha, const float *T_final, const int32_t *last, float *d_grid,
                              float *d_sh, cudaStream_t s) {
    const int ntiles = f.cam.ntx * f.cam.nty;
    const uint32_t *vals = f.vals[sorted_alt];
    cudaError_t e = cudaSuccess;
    if (f.n_vox > 0) e = cudaMemsetAsync(f.dcol, 0, sizeof(float) * 3 * (size_t)f.n_vox, s);
    if (e != cudaSuccess) return e;
    switch (f.K) {
        case 1: k_render_bwd<1><<<ntiles, kChunk, 0, s>>>(f, vals, d_rgb, d_depth, d_alpha, T_final, last, d_grid); break;
        case 2: k_render_bwd<2><<<ntiles, kChunk, 0, s>>>(f, vals, d_rgb, d_depth, d_alpha, T_final, last, d_grid); break;
        case 3: k_render_bwd<3><<<ntiles, kChunk, 0, s>>>(f, vals, d_rgb, d_depth, d_alpha, T_final, last, d_grid); break;
        default: return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (f.n_vox > 0) {
        k_voxel_bwd<<<(unsigned)((f.n_vox + 255) / 256), 256, 0, s>>>(f, d_sh);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace svr
