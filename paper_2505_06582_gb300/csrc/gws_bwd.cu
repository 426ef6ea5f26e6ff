// gws_bwd.cu -- backward of the splat: dL/d(mu, q, s, o, c) from G = dL/du_SLM (PyTorch's
// complex convention), for the order-invariant sum of Eq. 12 (and the depth-sorted weights
// with T_i held fixed; the cross terms through T_i are added by gws_tgrad kernels).
//
//   dL/dtheta = sum_f Re(conj(G(f)) d u_SLM(f) / dtheta)
//
// The spectra are recomputed, never stored.  A work item is a block of BB consecutive
// records of one wavelength (footprint order, so a block's footprints are alike).  The CTA
// walks the 64 x 48 frequency tiles of the block's footprint union; per tile it stages two
// per-pixel tables in shared memory with cp.async from copies laid out tile by tile
// (k_bwd_tables: (f_z - f0_z, log2 f_z - log2 |G|) and -arg G, padded past the grid so that a
// tile is one contiguous block per table, and a lane's two columns c and c + 32 of a row sit
// side by side for the packed f32x2 arithmetic): G enters in polar form, as a factor of the
// exponential and a shift of the phase, so conj(G) P0 costs no complex product.  It culls
// each record exactly (and where g = r3.f keeps one sign over the tile, folds that sign into
// the record's r3, so that its pixels skip their own) and hands the survivors to its warps
// through a shared counter; a warp takes one record over the tile (lane = column pair, rows
// in a loop, the phase re-anchored once per tile), accumulating 16 FP32 partial sums per
// column; these are reduced across the warp and merged per tile into 13 FP64 totals per
// record in shared memory:
//   TA = sum R a' d,  TB = sum R b' d,  TG = sum sign(g) Re(P0) f,  TI = sum I f,  SI = sum I,
// with P0 = conj(G) f_z^-1 2^-(a'^2+b'^2) e^{j phi},  R = |g| Re(P0),  I = |g| Im(P0),
// g = r3.f, d = f - f_r.  A record's totals are only touched by the warp holding it in the
// current tile, and tiles are visited in a fixed order, so the result is deterministic.
// Three CTAs share an SM (80 registers a thread): the kernel is bound by its FP32 work, and
// with 24 resident warps the FMA pipe stays busier than with 16 warps at more registers.
#include <type_traits>
#include <float.h>

#include "gws_prep.h"

namespace gws {

constexpr int BTW = 64, BTH = 48, BPX = BTW * BTH;
constexpr int BSEG = 48;     // rows per phase segment (one per tile: the phase is re-anchored at its middle row,
                             // so the rows' |t_y (dy - dy_s)| stays within 24 rows' worth)
constexpr int BQ = BPX / 2;  // column pairs per tile (entries of each table)
constexpr int BB = 128;   // records per work item
constexpr int BNT = 256;  // threads per CTA
constexpr int BCTA = 3;   // resident CTAs per SM (registers per thread: 65536 / (BCTA BNT))
constexpr int NTOT = 13;

static_assert(BTH % 2 == 0 && BQ % (2 * BNT) == 0, "tile tables are copied in whole 16-byte pieces per thread");

int bwd_block_size() { return BB; }
int bwd_ctas_per_sm() { return BCTA; }

struct TileConst {  // geometry of the current tile, computed once by thread 0
    double f0x, f0y, f0z, dz0;
    float x0, x1, y0, y1;
    float fzlo, fzhi;  // range of f_z over the tile's valid pixels (0 where evanescent)
    float dzt;         // bound on |f_z - 1/lambda| over them
    int c_lo, r_lo, c_ref, r_ref;
};

struct BwdShared {
    float4 t[BQ];   // [row][lane]: (dz(c), dz(c + 32), lw(c), lw(c + 32)), c = c_lo + lane, lw = log2(f_z / |G|)
    float2 ps[BQ];  // [row][lane]: (-arg G(c), -arg G(c + 32))
    Rec rec[BB];
    float4 sv[BB][4];
    int2 rows[BB];  // per surviving record: the tile rows [x, y] its footprint's bounding box reaches
    double tot[BB][NTOT];
    float red[BNT / 32][16];
    unsigned mask[BB / 32];
    signed char sgn[BB];     // per surviving record: the sign of g over the tile (0: it changes)
    unsigned char list[BB];  // the surviving records of the current tile, in record order
    int n_surv, next;        // their count; the next list entry a warp takes
    TileConst tc;
    int tx0, tx1, ty0, ty1;
    int item;
};
static_assert(BCTA * (sizeof(BwdShared) + 1024) <= 228 * 1024, "BCTA CTAs must fit an SM's shared memory");

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ bool ellipse_hits_rect_b(float e00, float e01, float e11, float x0, float x1, float y0,
                                                    float y1) {
    if (x0 <= 0.f && 0.f <= x1 && y0 <= 0.f && 0.f <= y1) return true;
    float best = 3.0e38f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float xe = k ? x1 : x0;
        const float ys = e11 > 0.f ? fminf(fmaxf(-e01 * xe / e11, y0), y1) : y0;
        best = fminf(best, e00 * xe * xe + 2.f * e01 * xe * ys + e11 * ys * ys);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float ye = k ? y1 : y0;
        const float xs = e00 > 0.f ? fminf(fmaxf(-e01 * ye / e00, x0), x1) : x0;
        best = fminf(best, e00 * xs * xs + 2.f * e01 * xs * ye + e11 * ye * ye);
    }
    return best <= 1.001f;
}

// Sum of v[0..15] over the warp; afterwards lane l holds the total of value l >> 1.
__device__ __forceinline__ float warp_transpose_reduce16(float v[16], int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool hi = lane & 16;
        const float send = hi ? v[i] : v[i + 8];
        const float keep = hi ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = lane & 8;
        const float send = hi ? v[i] : v[i + 4];
        const float keep = hi ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 4;
        const float send = hi ? v[i] : v[i + 2];
        const float keep = hi ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool hi = lane & 2;
        const float send = hi ? v[0] : v[1];
        const float keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// per-pixel table in the natural layout for tw x th tiles (the forward splat's prologue, the
// exact blend's and partial coherence's accumulation): (f_z - f0_z of the pixel's tile,
// log2(1 / f_z)); (0, -inf) where evanescent
__global__ void k_pixtab(int n_lambda, int H, int W, double dfx, double dfy, InvLam inv_lam, int tw, int th,
                         float2 *__restrict__ tab) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long hw = (long long)H * W;
    if (idx >= hw * n_lambda) return;
    const int l = (int)(idx / hw);
    const long long pix = idx % hw;
    const int r = (int)(pix / W), c = (int)(pix % W);
    const int tx = c / tw, ty = r / th;
    const int c_lo = tx * tw, r_lo = ty * th;
    const int c_hi = min(c_lo + tw, W) - 1, r_hi = min(r_lo + th, H) - 1;
    const double k2 = inv_lam.v[l] * inv_lam.v[l];
    int c_ref, r_ref;
    tile_ref(c_lo, c_hi, r_lo, r_hi, H, W, dfx, dfy, k2, c_ref, r_ref);
    const double f0x = (double)(c_ref - W / 2) * dfx, f0y = (double)(r_ref - H / 2) * dfy;
    const double f0z = sqrt(fmax(k2 - (f0x * f0x + f0y * f0y), 0.0));
    const double fx = (double)(c - W / 2) * dfx, fy = (double)(r - H / 2) * dfy;
    const double rho2 = fx * fx + fy * fy;
    float2 v;
    if (rho2 < k2) {
        const double fz = sqrt(k2 - rho2);
        v.x = (float)(fz - f0z);
        v.y = (float)(-log2(fz));
    } else {
        v.x = 0.f;
        v.y = -INFINITY;
    }
    tab[idx] = v;
}

// The backward's tile-major tables, one entry per (wavelength, tile, row, lane) holding the
// columns c = c_lo + lane and c + 32 of the row: t = (dz(c), dz(c + 32), lw(c), lw(c + 32)) with
// dz = f_z - f0_z (FP64, rounded) and lw = log2 f_z - log2 |G(f)|, and ps = -arg G, so that
//   conj(G) f_z^-1 2^-(a'^2 + b'^2) e^{j phi} = 2^-(a'^2 + b'^2 + lw) e^{j (phi + ps)}.
// Past the grid, where f is evanescent and where G = 0: dz = 0, lw = +inf (2^-inf = 0), ps = 0.
__global__ void k_bwd_tables(const float2 *__restrict__ G, int n_lambda, int H, int W, double dfx, double dfy,
                             InvLam inv_lam, int tiles_x, int tiles_y, float4 *__restrict__ tab,
                             float2 *__restrict__ ps) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per_l = (long long)tiles_x * tiles_y * BQ;
    if (idx >= per_l * n_lambda) return;
    const int l = (int)(idx / per_l);
    const long long rem = idx % per_l;
    const int t = (int)(rem / BQ), q = (int)(rem % BQ);
    const int tx = t % tiles_x, ty = t / tiles_x;
    const int c_lo = tx * BTW, r_lo = ty * BTH;
    const int r = r_lo + q / 32, c0 = c_lo + q % 32;
    const int c_hi = min(c_lo + BTW, W) - 1, r_hi = min(r_lo + BTH, H) - 1;
    const double k2 = inv_lam.v[l] * inv_lam.v[l];
    int c_ref, r_ref;
    tile_ref(c_lo, c_hi, r_lo, r_hi, H, W, dfx, dfy, k2, c_ref, r_ref);
    const double f0x = (double)(c_ref - W / 2) * dfx, f0y = (double)(r_ref - H / 2) * dfy;
    const double f0z = sqrt(fmax(k2 - (f0x * f0x + f0y * f0y), 0.0));
    float dz[2] = {0.f, 0.f}, lw[2] = {INFINITY, INFINITY}, ph[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = c0 + 32 * h;
        if (r >= H || c >= W) continue;
        const double fx = (double)(c - W / 2) * dfx, fy = (double)(r - H / 2) * dfy;
        const double rho2 = fx * fx + fy * fy;
        const float2 v = G[((size_t)l * H + r) * W + c];
        const float m = hypotf(v.x, v.y);
        if (rho2 < k2 && m > 0.f) {
            const double fz = sqrt(k2 - rho2);
            dz[h] = (float)(fz - f0z);
            lw[h] = (float)(log2(fz) - (double)log2f(m));
            ph[h] = -atan2f(v.y, v.x);
        }
    }
    tab[idx] = make_float4(dz[0], dz[1], lw[0], lw[1]);
    ps[idx] = make_float2(ph[0], ph[1]);
}

__global__ void __launch_bounds__(BNT, BCTA) k_splat_bwd(const __grid_constant__ BwdArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdShared &S = *reinterpret_cast<BwdShared *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n = A.segs.off[1];  // single scene

    for (;;) {
        if (tid == 0) S.item = atomicAdd(A.queue, 1);
        __syncthreads();
        const int it = S.item;
        if (it >= A.n_items) break;
        // wavelength-major: the CTAs in flight share one wavelength's tables in L2
        const int nblk = (int)((n + BB - 1) / BB);
        const int l = it / nblk, blk = it % nblk;
        if (!in_bounds(l < A.segs.n_lambda, A.status)) {  // checking build only
            __syncthreads();
            continue;
        }
        const long long seg_base = (long long)l * n;
        const long long k0 = (long long)blk * BB;
        const int nrec = (int)min((long long)BB, n - k0);
        const double inv_lam = A.inv_lam[l];
        const double k2 = inv_lam * inv_lam;
        {
            const float4 *src = reinterpret_cast<const float4 *>(A.rec + seg_base + k0);
            float4 *dst = reinterpret_cast<float4 *>(S.rec);
            for (int i = tid; i < nrec * 6; i += BNT) dst[i] = src[i];
        }
        for (int i = tid; i < BB * NTOT; i += BNT) (&S.tot[0][0])[i] = 0.0;
        if (tid == 0) {
            S.tx0 = A.tiles_x;
            S.tx1 = -1;
            S.ty0 = A.tiles_y;
            S.ty1 = -1;
        }
        __syncthreads();
        if (tid < nrec) {
            const Rec &r = S.rec[tid];
            const double det = (double)r.e00 * r.e11 - (double)r.e01 * r.e01;
            int c0 = 0, c1 = A.W - 1, q0 = 0, q1 = A.H - 1;
            if (det > 0.0) {
                const double hx = sqrt((double)r.e11 / det) * 1.001, hy = sqrt((double)r.e00 / det) * 1.001;
                const double cx = hx / A.dfx + 1.0, cy = hy / A.dfy + 1.0;
                c0 = (int)fmax(0.0, floor(A.W / 2 - cx));
                c1 = (int)fmin((double)(A.W - 1), ceil(A.W / 2 + cx));
                q0 = (int)fmax(0.0, floor(A.H / 2 - cy));
                q1 = (int)fmin((double)(A.H - 1), ceil(A.H / 2 + cy));
            }
            atomicMin(&S.tx0, c0 / BTW);
            atomicMax(&S.tx1, c1 / BTW);
            atomicMin(&S.ty0, q0 / BTH);
            atomicMax(&S.ty1, q1 / BTH);
        }
        __syncthreads();
        const int ntx = S.tx1 - S.tx0 + 1, nty = S.ty1 - S.ty0 + 1;
        const int n_t = (ntx > 0 && nty > 0) ? ntx * nty : 0;
        const size_t ntiles = (size_t)A.tiles_x * A.tiles_y;
        const float4 *tsl = A.tab + (size_t)l * ntiles * BQ;
        const float2 *psl = A.ps + (size_t)l * ntiles * BQ;

        // one buffer per table (the tables of a 64 x 48 tile take 36 KB, so that three CTAs of 80
        // registers a thread fit an SM): the copy of tile t overlaps its cull; the other resident
        // CTAs cover the rest of the wait
        for (int t = 0; t < n_t; ++t) {
            {
                size_t tile = (size_t)(S.ty0 + t / ntx) * A.tiles_x + (S.tx0 + t % ntx);
                if (!in_bounds(S.tx0 >= 0 && S.ty0 >= 0 && S.tx1 < A.tiles_x && S.ty1 < A.tiles_y && tile < ntiles,
                               A.status))
                    tile = 0;
#pragma unroll
                for (int i = 0; i < BQ / BNT; ++i) {
                    const int e = tid + BNT * i;
                    cp_async16(&S.t[e], tsl + tile * BQ + e);
                }
#pragma unroll
                for (int i = 0; i < BQ / (2 * BNT); ++i) {  // two float2 per 16-byte copy
                    const int e = 2 * (tid + BNT * i);
                    cp_async16(&S.ps[e], psl + tile * BQ + e);
                }
                cp_async_commit();
            }
            if (tid == 0) {
                TileConst &T = S.tc;
                const int tx = S.tx0 + t % ntx, ty = S.ty0 + t / ntx;
                T.c_lo = tx * BTW;
                T.r_lo = ty * BTH;
                const int c_hi = min(T.c_lo + BTW, A.W) - 1, r_hi = min(T.r_lo + BTH, A.H) - 1;
                tile_ref(T.c_lo, c_hi, T.r_lo, r_hi, A.H, A.W, A.dfx, A.dfy, k2, T.c_ref, T.r_ref);
                T.f0x = (double)(T.c_ref - A.W / 2) * A.dfx;
                T.f0y = (double)(T.r_ref - A.H / 2) * A.dfy;
                T.f0z = sqrt(fmax(k2 - (T.f0x * T.f0x + T.f0y * T.f0y), 0.0));
                T.dz0 = T.f0z - inv_lam;
                T.x0 = (float)((double)(T.c_lo - A.W / 2) * A.dfx);
                T.x1 = (float)((double)(c_hi - A.W / 2) * A.dfx);
                T.y0 = (float)((double)(T.r_lo - A.H / 2) * A.dfy);
                T.y1 = (float)((double)(r_hi - A.H / 2) * A.dfy);
                fz_range((double)(T.c_lo - A.W / 2) * A.dfx, (double)(c_hi - A.W / 2) * A.dfx,
                         (double)(T.r_lo - A.H / 2) * A.dfy, (double)(r_hi - A.H / 2) * A.dfy, k2, T.fzlo, T.fzhi);
                T.dzt = (float)dz_far((double)(T.c_lo - A.W / 2) * A.dfx, (double)(c_hi - A.W / 2) * A.dfx,
                                      (double)(T.r_lo - A.H / 2) * A.dfy, (double)(r_hi - A.H / 2) * A.dfy, inv_lam);
            }
            __syncthreads();
            const int c_lo = S.tc.c_lo, r_lo = S.tc.r_lo, c_ref = S.tc.c_ref, r_ref = S.tc.r_ref;
            // cull + per-(record, tile) scalars
            if (tid < BB) {
                bool pass = false;
                if (tid < nrec) {
                    const Rec &r = S.rec[tid];
                    const double f0x = S.tc.f0x, f0y = S.tc.f0y, f0z = S.tc.f0z, dz0 = S.tc.dz0;
                    // the footprint for this tile's bound on |d_z| (within the grid-wide one)
                    const float sc = footprint_scale(A.dzmax[l], S.tc.dzt, r.wz);
                    const float e00 = r.e00 * sc, e01 = r.e01 * sc, e11 = r.e11 * sc;
                    pass = ellipse_hits_rect_b(e00, e01, e11, S.tc.x0, S.tc.x1, S.tc.y0, S.tc.y1);
                    if (pass) {
                        // rows of the tile inside the footprint's bounding box
                        const float det = e00 * e11 - e01 * e01;
                        int rlo = 0, rhi = BTH - 1;
                        if (det > 0.f) {
                            const float hy = sqrtf(e00 / det) * 1.001f + 1e-3f * (float)A.dfy;
                            const float dfyf = (float)A.dfy;
                            rlo = max(0, (int)ceilf((-hy - S.tc.y0) / dfyf));
                            rhi = min(BTH - 1, (int)floorf((hy - S.tc.y0) / dfyf));
                        }
                        S.rows[tid] = make_int2(rlo, rhi);
                        double cyc = -(f0x * r.mux + f0y * r.muy + f0z * r.muz);
                        if (A.phase_match) cyc += r.muz * inv_lam;
                        cyc -= rint(cyc);
                        cyc *= kTwoPi;
                        const float fxf = (float)f0x, fyf = (float)f0y, fzf = (float)f0z, dzf = (float)dz0;
                        S.sv[tid][0] = make_float4(r.r1x, r.r1y, r.r1z, fmaf(r.r1z, dzf, fmaf(r.r1y, fyf, r.r1x * fxf)));
                        S.sv[tid][1] = make_float4(r.r2x, r.r2y, r.r2z, fmaf(r.r2z, dzf, fmaf(r.r2y, fyf, r.r2x * fxf)));
                        // where g keeps one sign over the tile it is folded into r3 (g' = |g|), so that the
                        // pixels need no sign of their own; the Rg moments are multiplied back by it
                        const int sg =
                            sign_over_box(r.r3x, r.r3y, r.r3z, S.tc.x0, S.tc.x1, S.tc.y0, S.tc.y1, S.tc.fzlo, S.tc.fzhi);
                        const float sf = sg < 0 ? -1.f : 1.f;
                        S.sgn[tid] = (signed char)sg;
                        S.sv[tid][2] = make_float4(sf * r.r3x, sf * r.r3y, sf * r.r3z,
                                                   sf * fmaf(r.r3z, fzf, fmaf(r.r3y, fyf, r.r3x * fxf)));
                        S.sv[tid][3] = make_float4(r.mx, r.my, r.mz, (float)cyc);
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, pass);
                if (lane == 0) S.mask[warp] = bal;
            }
            __syncthreads();
            if (tid < BB) {  // compact the survivors; warps then take them one by one
                int before = 0;
                for (int w = 0; w < tid / 32; ++w) before += __popc(S.mask[w]);
                const unsigned m = S.mask[tid / 32];
                if ((m >> lane) & 1u) S.list[before + __popc(m & ((1u << lane) - 1u))] = (unsigned char)tid;
                if (tid == BB - 1) {
                    S.n_surv = before + __popc(m);
                    S.next = 0;
                }
            }
            cp_async_wait0();
            __syncthreads();
            const float dfxf = (float)A.dfx, dfyf = (float)A.dfy;
            const float dx0 = (float)(c_lo + lane - c_ref) * dfxf;  // the lane's columns c and c + 32
            const float dx1 = (float)(c_lo + lane + 32 - c_ref) * dfxf;
            const float dyb = (float)(r_lo - r_ref) * dfyf;
            const int n_surv = S.n_surv;
            for (;;) {
                int j = 0;
                if (lane == 0) j = atomicAdd(&S.next, 1);
                j = __shfl_sync(0xffffffffu, j, 0);
                if (j >= n_surv) break;
                const int k = S.list[j];
                if (!in_bounds(k < nrec, A.status)) continue;
                const int2 rr = S.rows[k];
                const int row_lo = rr.x, row_hi = rr.y;
                if (!in_bounds(row_lo >= 0 && row_hi < BTH, A.status)) continue;
                const float4 Ar = S.sv[k][0], Br = S.sv[k][1], Gr = S.sv[k][2], Mr = S.sv[k][3];
                const float2 ac = make_float2(fmaf(Ar.x, dx0, Ar.w), fmaf(Ar.x, dx1, Ar.w));
                const float2 bc = make_float2(fmaf(Br.x, dx0, Br.w), fmaf(Br.x, dx1, Br.w));
                const float2 gc = make_float2(fmaf(Gr.x, dx0, Gr.w), fmaf(Gr.x, dx1, Gr.w));
                // the phase at the lane's two columns on the tile's reference row (FP32 from the
                // reduced FP64 anchor); per segment of BSEG rows it is moved to the segment's middle
                // row and reduced to [-pi, pi] (t / 2 pi + 1.5 2^23, minus 1.5 2^23: the nearest turn
                // count), and the rows' |t_y (dy - dy_s)| + |t_z dz| are added unreduced before sin/cos
                // (the argument error of sin.approx grows like 1.2e-7 |t|)
                const float2 tc = make_float2(fmaf(Mr.x, dx0, Mr.w), fmaf(Mr.x, dx1, Mr.w));
                const float2 ay = pair(Ar.y), az = pair(Ar.z), by = pair(Br.y), bz = pair(Br.z);
                const float2 gy = pair(Gr.y), gz = pair(Gr.z), ty = pair(Mr.y), tz = pair(Mr.z);
                float2 sp[4], sz[4], sy[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) sp[u] = sz[u] = sy[u] = pair(0.f);
                const int sgn = S.sgn[k];
                // SIGNED: g changes sign inside the tile and each pixel takes its own
                auto rows = [&](auto signed_tag) {
                    constexpr bool SIGNED = decltype(signed_tag)::value;
                    for (int seg = row_lo / BSEG; seg <= row_hi / BSEG; ++seg) {
                        const int s_lo = max(row_lo, seg * BSEG), s_hi = min(row_hi, seg * BSEG + BSEG - 1);
                        const float dys = fmaf((float)(seg * BSEG + BSEG / 2), dfyf, dyb);  // dy of the middle row
                        float2 ts = __ffma2_rn(ty, pair(dys), tc);
                        {
                            const float2 kt = __fadd2_rn(__ffma2_rn(ts, pair(0.15915494309189535f), pair(12582912.0f)),
                                                         pair(-12582912.0f));
                            ts = __ffma2_rn(kt, pair(-6.28318530717958647692f), ts);
                        }
                        // t_y dy + ts is the reduced phase plus t_y (dy - dy_s): one rounding of t_y dy_s here
                        ts = __ffma2_rn(ty, pair(-dys), ts);
                        // one row = the lane's two columns as one f32x2 pair; up to 24 rows in flight
#pragma unroll 24
                        for (int row = s_lo; row <= s_hi; ++row) {
                            const float2 dy = pair(fmaf((float)row, dfyf, dyb));
                            const float4 T4 = S.t[32 * row + lane];
                            const float2 ps = S.ps[32 * row + lane];
                            const float2 dz = make_float2(T4.x, T4.y), lw = make_float2(T4.z, T4.w);
                            const float2 a = __ffma2_rn(az, dz, __ffma2_rn(ay, dy, ac));
                            const float2 b = __ffma2_rn(bz, dz, __ffma2_rn(by, dy, bc));
                            const float2 g = __ffma2_rn(gz, dz, __ffma2_rn(gy, dy, gc));
                            const float2 ang = __ffma2_rn(tz, dz, __fadd2_rn(__ffma2_rn(ty, dy, ts), ps));  // phi - arg G
                            const float2 uq = __ffma2_rn(a, a, __ffma2_rn(b, b, lw));  // a'^2 + b'^2 + log2(f_z / |G|)
                            float2 es = make_float2(ex2_approx(-uq.x), ex2_approx(-uq.y));
                            if constexpr (SIGNED) es = make_float2(with_sign_of(es.x, g.x), with_sign_of(es.y, g.y));
                            // sign(g) P0 = sign(g) conj(G) f_z^-1 2^-(a'^2+b'^2) e^{j phi} = Rg + j Pi
                            const float2 Rg = __fmul2_rn(es, make_float2(cos_approx(ang.x), cos_approx(ang.y)));
                            const float2 Pi = __fmul2_rn(es, make_float2(sin_approx(ang.x), sin_approx(ang.y)));
                            const float2 R = __fmul2_rn(g, Rg), I = __fmul2_rn(g, Pi);  // |g| Re P0, |g| Im P0
                            const float2 X[4] = {__fmul2_rn(R, a), __fmul2_rn(R, b), Rg, I};
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                sp[u] = __fadd2_rn(sp[u], X[u]);
                                sy[u] = __ffma2_rn(X[u], dy, sy[u]);
                                sz[u] = __ffma2_rn(X[u], dz, sz[u]);
                            }
                        }
                    }
                };
                if (sgn == 0) {
                    rows(std::true_type{});
                } else {
                    rows(std::false_type{});
                    if (sgn < 0) {  // back to sign(g) P0 for the Rg moments
                        sp[2] = __fmul2_rn(sp[2], pair(-1.f));
                        sy[2] = __fmul2_rn(sy[2], pair(-1.f));
                        sz[2] = __fmul2_rn(sz[2], pair(-1.f));
                    }
                }
                float v[16];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    v[4 * u + 0] = sp[u].x + sp[u].y;
                    v[4 * u + 1] = fmaf(dx0, sp[u].x, dx1 * sp[u].y);
                    v[4 * u + 2] = sy[u].x + sy[u].y;
                    v[4 * u + 3] = sz[u].x + sz[u].y;
                }
                const float tot = warp_transpose_reduce16(v, lane);
                if ((lane & 1) == 0) S.red[warp][lane >> 1] = tot;
                __syncwarp();
                if (lane < NTOT) {
                    double add;
                    if (lane == 12) {
                        add = (double)S.red[warp][12];
                    } else {
                        const int vec = lane / 3, comp = lane % 3;
                        const double ref = comp == 0 ? S.tc.f0x : (comp == 1 ? S.tc.f0y : (vec < 2 ? S.tc.dz0 : S.tc.f0z));
                        add = ref * (double)S.red[warp][4 * vec] + (double)S.red[warp][4 * vec + 1 + comp];
                    }
                    S.tot[k][lane] += add;
                }
                __syncwarp();
            }
            __syncthreads();
        }
        cp_async_wait0();
        __syncthreads();
        for (int i = tid; i < nrec * NTOT; i += BNT)
            A.acc[(size_t)(seg_base + k0 + i / NTOT) * NTOT + i % NTOT] = S.tot[i / NTOT][i % NTOT];
        __syncthreads();
    }
}

// dL/d(parameters) per Gaussian from the per-(Gaussian, wavelength) totals
__global__ void k_grad_assemble(const GPre *__restrict__ gp, const float *__restrict__ ampc,
                                const double *__restrict__ T_g, const int *__restrict__ invrec,
                                const double *__restrict__ acc, const float *__restrict__ quat_in, long long n, int L,
                                GradArgs G) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const GPre &P = gp[g];
    double r1[3], r2[3], r3[3];
    quat_cols<double>(P.q, r1, r2, r3);
    const double su = P.su, sv = P.sv, o = P.o;
    const double T = T_g ? T_g[g] : 1.0;
    const double ln2 = 0.69314718055994530942;
    double dmu[3] = {0, 0, 0}, G1[3] = {0, 0, 0}, G2[3] = {0, 0, 0}, G3[3] = {0, 0, 0};
    double dsu = 0, dsv = 0, dop = 0, dT = 0;
    for (int l = 0; l < L; ++l) {
        const int ri = invrec[g * L + l];
        if (!in_bounds(ri >= 0 && (long long)ri < n * L, G.status)) continue;
        const double *t = acc + (size_t)ri * NTOT;
        const double c = ampc[g * L + l];
        const double Wl = kTwoPi * su * sv * c * o * T;
        double dr1p[3], dr2p[3], dW = 0;
        for (int k = 0; k < 3; ++k) {
            dr1p[k] = -2.0 * ln2 * Wl * t[k];
            dr2p[k] = -2.0 * ln2 * Wl * t[3 + k];
            G3[k] += Wl * t[6 + k];
            dW += r3[k] * t[6 + k];
            dmu[k] += kTwoPi * Wl * t[9 + k];
        }
        if (G.phase_match) dmu[2] -= kTwoPi * G.inv_lam[l] * Wl * t[12];
        const double ku = kKappa * su, kv = kKappa * sv;
        for (int k = 0; k < 3; ++k) {
            G1[k] += ku * dr1p[k];
            G2[k] += kv * dr2p[k];
        }
        dsu += kKappa * (r1[0] * dr1p[0] + r1[1] * dr1p[1] + r1[2] * dr1p[2]);
        dsv += kKappa * (r2[0] * dr2p[0] + r2[1] * dr2p[1] + r2[2] * dr2p[2]);
        const double base = kTwoPi * su * sv;  // W = base * c * o * T
        dsu += kTwoPi * sv * c * o * T * dW;
        dsv += kTwoPi * su * c * o * T * dW;
        G.amp[g * L + l] = (float)(base * o * T * dW);
        dop += base * c * T * dW;
        dT += base * c * o * dW;
    }
    // quaternion: R(qhat), qhat = q / |q|
    const double w = P.q[0], x = P.q[1], y = P.q[2], z = P.q[3];
    const double dr1[4][3] = {{0, 2 * z, -2 * y}, {0, 2 * y, 2 * z}, {-4 * y, 2 * x, -2 * w}, {-4 * z, 2 * w, 2 * x}};
    const double dr2[4][3] = {{-2 * z, 0, 2 * x}, {2 * y, -4 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, -4 * z, 2 * y}};
    const double dr3[4][3] = {{2 * y, -2 * x, 0}, {2 * z, -2 * w, -4 * x}, {2 * w, 2 * z, -4 * y}, {2 * x, 2 * y, 0}};
    double gh[4];
    for (int m = 0; m < 4; ++m) {
        gh[m] = 0;
        for (int k = 0; k < 3; ++k) gh[m] += G1[k] * dr1[m][k] + G2[k] * dr2[m][k] + G3[k] * dr3[m][k];
    }
    const double qi[4] = {quat_in[4 * g], quat_in[4 * g + 1], quat_in[4 * g + 2], quat_in[4 * g + 3]};
    const double qn = sqrt(qi[0] * qi[0] + qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]);
    const double proj = gh[0] * w + gh[1] * x + gh[2] * y + gh[3] * z;
    const double qh[4] = {w, x, y, z};
    for (int m = 0; m < 4; ++m) G.quat[4 * g + m] = (float)((gh[m] - proj * qh[m]) / qn);
    for (int k = 0; k < 3; ++k) G.mean[3 * g + k] = dmu[k];
    G.scale[2 * g] = (float)dsu;
    G.scale[2 * g + 1] = (float)dsv;
    G.opacity[g] = (float)dop;
    if (G.dT) G.dT[g] = dT;
}

cudaError_t launch_pixtab(int n_lambda, int H, int W, double dfx, double dfy, const InvLam &il, int tw, int th,
                          float2 *tab, cudaStream_t s) {
    const long long n = (long long)n_lambda * H * W;
    k_pixtab<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n_lambda, H, W, dfx, dfy, il, tw, th, tab);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_bwd_tables(int n_lambda, int H, int W, double dfx, double dfy, const InvLam &il, const float2 *G,
                              float4 *tab, float2 *ps, cudaStream_t s) {
    const int tx = bwd_tiles_x(W), ty = bwd_tiles_y(H);
    const long long n = (long long)n_lambda * tx * ty * BQ;
    k_bwd_tables<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(G, n_lambda, H, W, dfx, dfy, il, tx, ty, tab, ps);
    count_launches(1);
    return cudaGetLastError();
}

int bwd_tiles_x(int W) { return (W + BTW - 1) / BTW; }
int bwd_tiles_y(int H) { return (H + BTH - 1) / BTH; }
size_t bwd_table_bytes(int n_lambda, int H, int W) {
    return sizeof(float4) * (size_t)n_lambda * bwd_tiles_x(W) * bwd_tiles_y(H) * BQ;
}

cudaError_t prepare_bwd_kernels() {
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_splat_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BwdShared));
    // BCTA CTAs' shared memory per SM needs the largest shared-memory carveout
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_splat_bwd, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

cudaError_t launch_splat_bwd(const BwdArgs &a, int grid, cudaStream_t s) {
    const size_t smem = sizeof(BwdShared);
    cudaError_t e = prepare_bwd_kernels();
    if (e != cudaSuccess) return e;
    k_splat_bwd<<<grid, BNT, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_grad_assemble(const GPre *gp, const float *ampc, const double *T_g, const int *invrec,
                                 const double *acc, const float *quat_in, long long n, int L, const GradArgs &G,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_grad_assemble<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(gp, ampc, T_g, invrec, acc, quat_in, n, L, G);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gws
