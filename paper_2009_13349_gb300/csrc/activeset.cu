// Active-set construction (Sec. 6, Algorithm 3) for GB300 (sm_103a): a
// swept-box broad phase on a uniform grid, the CCD of every candidate
// through the segmented batch of ccd.cu, and the compaction of the
// candidates that collide.
//
// Broad phase (the paper names it only; this is its plain definition): every
// vertex-face pair (v, f), v not a vertex of f, and every edge-edge pair
// (a, b), a < b, without a shared vertex, whose swept boxes overlap.  A swept
// box is the per-axis min / max of the primitive's vertices at both times,
// minus / plus a margin r; boxes overlap when lo_1 <= hi_2 and lo_2 <= hi_1
// on every axis.
//
// Grid: the cell edge h is a power of two >= 1.01 times the largest box
// extent, so cell(x) = floor((x - o) / h) is exact up to the rounding of
// x - o and every box covers at most two cells per axis.  Each primitive
// writes one (cell key, id) entry per covered cell into 8 fixed slots; the
// entries are sorted by key (CUB radix sort, library code); one thread per
// entry tests it against the later entries of its cell.  A pair is emitted
// only in the cell that holds the lower corner max(lo_1, lo_2) of the two
// boxes' intersection, which both boxes cover, so it is emitted exactly once.
// Candidates are then sorted by (first id, second id), a deterministic order.

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <cstdint>
#include <cstring>

#include "ccd.h"

namespace {

constexpr int BP_SLOTS = 8;
constexpr unsigned long long BP_NONE = ~0ull;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

__device__ __forceinline__ long long okey(double x)   // order-preserving signed key
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

struct BpScene {
    long long lo_key[3];           // min over boxes of lo, order-preserving keys
    long long hi_key[3];           // max over boxes of hi
    unsigned long long ext_bits;   // max box extent (>= 0, raw bits order)
    unsigned long long gamma_bits[3];   // max(1, max |x|) per axis, both times
    unsigned long long vf_count, ee_count;
};

// primitive p: vertex (p < nv), face (p < nv + nf) or edge
__device__ __forceinline__ int prim_points(long long p, long long nv, long long nf,
                                           const int *faces, const int *edges, int ids[3])
{
    if (p < nv) { ids[0] = (int)p; return 1; }
    if (p < nv + nf) {
        const long long f = p - nv;
        ids[0] = faces[3 * f]; ids[1] = faces[3 * f + 1]; ids[2] = faces[3 * f + 2];
        return 3;
    }
    const long long e = p - nv - nf;
    ids[0] = edges[2 * e]; ids[1] = edges[2 * e + 1];
    return 2;
}

__global__ void bp_init_kernel(BpScene *sc)
{
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; ++c) {
            sc->lo_key[c] = 0x7fffffffffffffffLL;
            sc->hi_key[c] = (long long)0x8000000000000000ULL;
            sc->gamma_bits[c] = (unsigned long long)__double_as_longlong(1.0);
        }
        sc->ext_bits = 0ull;
        sc->vf_count = sc->ee_count = 0ull;
    }
}

// gamma_c = max(1, max over vertices and both times of |x_c|)
__global__ void bp_gamma_kernel(const double *x0, const double *x1, long long nv, BpScene *sc)
{
    unsigned long long g[3] = {0ull, 0ull, 0ull};
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (long long)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) {
            const unsigned long long a = (unsigned long long)__double_as_longlong(fabs(x0[3 * v + c]));
            const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(x1[3 * v + c]));
            g[c] = max(g[c], max(a, b));
        }
    for (int c = 0; c < 3; ++c) {
        for (int o = 16; o; o >>= 1) g[c] = max(g[c], (unsigned long long)__shfl_xor_sync(0xffffffffu, g[c], o));
        if ((threadIdx.x & 31) == 0) atomicMax(&sc->gamma_bits[c], g[c]);
    }
}

__global__ void bp_boxes_kernel(const double *x0, const double *x1, long long nv, long long nf,
                                long long ne, const int *faces, const int *edges, double r,
                                double *boxes, BpScene *sc)
{
    const long long np = nv + nf + ne;
    long long lo_k[3] = {0x7fffffffffffffffLL, 0x7fffffffffffffffLL, 0x7fffffffffffffffLL};
    long long hi_k[3] = {(long long)0x8000000000000000ULL, (long long)0x8000000000000000ULL,
                         (long long)0x8000000000000000ULL};
    unsigned long long ext = 0ull;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (long long)gridDim.x * blockDim.x) {
        int ids[3];
        const int k = prim_points(p, nv, nf, faces, edges, ids);
        for (int c = 0; c < 3; ++c) {
            double lo = x0[3 * ids[0] + c], hi = lo;
            for (int j = 0; j < k; ++j) {
                const double a = x0[3 * ids[j] + c], b = x1[3 * ids[j] + c];
                lo = fmin(lo, fmin(a, b));
                hi = fmax(hi, fmax(a, b));
            }
            lo = __dsub_rn(lo, r);
            hi = __dadd_rn(hi, r);
            boxes[6 * p + c] = lo;
            boxes[6 * p + 3 + c] = hi;
            lo_k[c] = min(lo_k[c], okey(lo));
            hi_k[c] = max(hi_k[c], okey(hi));
            ext = max(ext, (unsigned long long)__double_as_longlong(__dsub_rn(hi, lo)));
        }
    }
    for (int c = 0; c < 3; ++c) {
        for (int o = 16; o; o >>= 1) {
            lo_k[c] = min(lo_k[c], (long long)__shfl_xor_sync(0xffffffffu, lo_k[c], o));
            hi_k[c] = max(hi_k[c], (long long)__shfl_xor_sync(0xffffffffu, hi_k[c], o));
        }
    }
    for (int o = 16; o; o >>= 1) ext = max(ext, (unsigned long long)__shfl_xor_sync(0xffffffffu, ext, o));
    if ((threadIdx.x & 31) == 0) {
        for (int c = 0; c < 3; ++c) {
            atomicMin(&sc->lo_key[c], lo_k[c]);
            atomicMax(&sc->hi_key[c], hi_k[c]);
        }
        atomicMax(&sc->ext_bits, ext);
    }
}

struct Grid {
    double o[3];
    double h;
};

__device__ __forceinline__ long long cell_of(double x, double o, double h)
{
    return (long long)floor(__ddiv_rn(__dsub_rn(x, o), h));
}

__device__ __forceinline__ unsigned long long cell_key(long long ix, long long iy, long long iz)
{
    return ((unsigned long long)ix << 42) | ((unsigned long long)iy << 21) | (unsigned long long)iz;
}

__global__ void bp_entries_kernel(const double *boxes, long long np, Grid g,
                                  unsigned long long *keys, int *vals)
{
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (long long)gridDim.x * blockDim.x) {
        long long c0[3], c1[3];
        for (int c = 0; c < 3; ++c) {
            c0[c] = cell_of(boxes[6 * p + c], g.o[c], g.h);
            c1[c] = cell_of(boxes[6 * p + 3 + c], g.o[c], g.h);
            if (c1[c] > c0[c] + 1) c1[c] = c0[c] + 1;   // unreachable for h >= 1.01 extent
        }
        int s = 0;
        for (long long ix = c0[0]; ix <= c1[0]; ++ix)
            for (long long iy = c0[1]; iy <= c1[1]; ++iy)
                for (long long iz = c0[2]; iz <= c1[2]; ++iz) {
                    keys[BP_SLOTS * p + s] = cell_key(ix, iy, iz);
                    vals[BP_SLOTS * p + s] = (int)p;
                    ++s;
                }
        for (; s < BP_SLOTS; ++s) {
            keys[BP_SLOTS * p + s] = BP_NONE;
            vals[BP_SLOTS * p + s] = -1;
        }
    }
}

__device__ __forceinline__ bool boxes_overlap(const double *a, const double *b)
{
    return a[0] <= b[3] && b[0] <= a[3] && a[1] <= b[4] && b[1] <= a[4] && a[2] <= b[5] &&
           b[2] <= a[5];
}

__global__ void bp_pairs_kernel(const unsigned long long *keys, const int *vals, long long m,
                                const double *boxes, long long nv, long long nf,
                                const int *faces, const int *edges, Grid g,
                                unsigned long long *vf_keys, long long cap_vf,
                                unsigned long long *ee_keys, long long cap_ee, BpScene *sc)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
        if (key == BP_NONE) continue;
        const long long pa = vals[i];
        const int ta = pa < nv ? 0 : (pa < nv + nf ? 1 : 2);
        const double *ba = boxes + 6 * pa;
        for (long long j = i + 1; j < m && keys[j] == key; ++j) {
            const long long pb = vals[j];
            const int tb = pb < nv ? 0 : (pb < nv + nf ? 1 : 2);
            const bool vf = (ta == 0 && tb == 1) || (ta == 1 && tb == 0);
            const bool ee = ta == 2 && tb == 2;
            if (!vf && !ee) continue;
            const double *bb = boxes + 6 * pb;
            if (!boxes_overlap(ba, bb)) continue;
            // the lower corner of the intersection decides the reporting cell
            const unsigned long long here =
                cell_key(cell_of(fmax(ba[0], bb[0]), g.o[0], g.h),
                         cell_of(fmax(ba[1], bb[1]), g.o[1], g.h),
                         cell_of(fmax(ba[2], bb[2]), g.o[2], g.h));
            if (here != key) continue;
            if (vf) {
                const long long v = ta == 0 ? pa : pb, f = (ta == 0 ? pb : pa) - nv;
                if (faces[3 * f] == v || faces[3 * f + 1] == v || faces[3 * f + 2] == v) continue;
                const unsigned long long slot = atomicAdd(&sc->vf_count, 1ull);
                if ((long long)slot < cap_vf)
                    vf_keys[slot] = ((unsigned long long)v << 32) | (unsigned long long)f;
            } else {
                long long a = pa - nv - nf, b = pb - nv - nf;
                if (a > b) { const long long t = a; a = b; b = t; }
                const int a0 = edges[2 * a], a1 = edges[2 * a + 1];
                const int b0 = edges[2 * b], b1 = edges[2 * b + 1];
                if (a0 == b0 || a0 == b1 || a1 == b0 || a1 == b1) continue;
                const unsigned long long slot = atomicAdd(&sc->ee_count, 1ull);
                if ((long long)slot < cap_ee)
                    ee_keys[slot] = ((unsigned long long)a << 32) | (unsigned long long)b;
            }
        }
    }
}

__global__ void bp_unpack_kernel(const unsigned long long *keys, long long n, int *pairs)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        pairs[2 * i] = (int)(keys[i] >> 32);
        pairs[2 * i + 1] = (int)(keys[i] & 0xffffffffull);
    }
}

// query columns: VF (p, v1, v2, v3), EE (p1, p2, p3, p4), at t0 then t1
__global__ void as_gather_kernel(const double *x0, const double *x1, const int *faces,
                                 const int *edges, const int *vf_pairs, long long n_vf,
                                 const int *ee_pairs, long long n_ee, double *soa)
{
    const long long n = n_vf + n_ee;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int ids[4];
        if (i < n_vf) {
            const int f = vf_pairs[2 * i + 1];
            ids[0] = vf_pairs[2 * i];
            ids[1] = faces[3 * f]; ids[2] = faces[3 * f + 1]; ids[3] = faces[3 * f + 2];
        } else {
            const long long j = i - n_vf;
            const int a = ee_pairs[2 * j], b = ee_pairs[2 * j + 1];
            ids[0] = edges[2 * a]; ids[1] = edges[2 * a + 1];
            ids[2] = edges[2 * b]; ids[3] = edges[2 * b + 1];
        }
        for (int k = 0; k < 4; ++k)
            for (int c = 0; c < 3; ++c) {
                soa[(size_t)(3 * k + c) * n + i] = x0[3 * ids[k] + c];
                soa[(size_t)(12 + 3 * k + c) * n + i] = x1[3 * ids[k] + c];
            }
    }
}

__global__ void as_flags_kernel(const uint8_t *collides, long long n, int *flags)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        flags[i] = collides[i] ? 1 : 0;
}

__global__ void as_scatter_kernel(const int *flags, const int *pos, long long n, long long n_vf,
                                  const int *vf_pairs, const int *ee_pairs, const double *toi,
                                  int *out_kind, int *out_pairs, double *out_toi)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (!flags[i]) continue;
        const int o = pos[i];
        const bool vf = i < n_vf;
        const int *pr = vf ? vf_pairs + 2 * i : ee_pairs + 2 * (i - n_vf);
        out_kind[o] = vf ? CCD_KIND_VF : CCD_KIND_EE;
        out_pairs[2 * o] = pr[0];
        out_pairs[2 * o + 1] = pr[1];
        out_toi[o] = toi[i];
    }
}

int grid_blocks(long long n)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long b = (n + 255) / 256;
    const long long cap = 8LL * (sms > 0 ? sms : 1);
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

// broad-phase workspace layout
struct BpLayout {
    size_t scene, boxes, keys0, keys1, vals0, vals1, cand0, cand1, cand2, temp, total;
    size_t temp_bytes;
};

bool bp_layout(long long nv, long long nf, long long ne, long long cap_vf, long long cap_ee,
               BpLayout *L)
{
    const long long np = nv + nf + ne, m = BP_SLOTS * np;
    const long long cap = cap_vf > cap_ee ? cap_vf : cap_ee;
    size_t t1 = 0, t2 = 0;
    if (cub::DeviceRadixSort::SortPairs(nullptr, t1, (unsigned long long *)nullptr,
                                        (unsigned long long *)nullptr, (int *)nullptr,
                                        (int *)nullptr, (int)(m > 0 ? m : 1)) != cudaSuccess ||
        cub::DeviceRadixSort::SortKeys(nullptr, t2, (unsigned long long *)nullptr,
                                       (unsigned long long *)nullptr,
                                       (int)(cap > 0 ? cap : 1)) != cudaSuccess)
        return false;
    size_t off = 0;
    L->scene = off; off = al256(off + sizeof(BpScene));
    L->boxes = off; off = al256(off + sizeof(double) * 6 * (size_t)np);
    L->keys0 = off; off = al256(off + sizeof(unsigned long long) * (size_t)m);
    L->keys1 = off; off = al256(off + sizeof(unsigned long long) * (size_t)m);
    L->vals0 = off; off = al256(off + sizeof(int) * (size_t)m);
    L->vals1 = off; off = al256(off + sizeof(int) * (size_t)m);
    L->cand0 = off; off = al256(off + sizeof(unsigned long long) * (size_t)cap);
    L->cand1 = off; off = al256(off + sizeof(unsigned long long) * (size_t)cap);
    L->cand2 = off; off = al256(off + sizeof(unsigned long long) * (size_t)cap);
    L->temp_bytes = t1 > t2 ? t1 : t2;
    L->temp = off; off = al256(off + L->temp_bytes);
    L->total = off;
    return true;
}

// eps of the scene (Sec. 6, the bounds of all the vertices of the
// simulation): gamma_c = max(1, max |x_c| over every vertex at both times),
// eps_c = K ((gamma_c gamma_c) gamma_c), K of Eq. ccd-error per kind.
// Synchronizes the stream.
ccd_status scene_eps(const double *x0, const double *x1, long long nv, BpScene *sc,
                     double eps[6], cudaStream_t st)
{
    bp_init_kernel<<<1, 32, 0, st>>>(sc);
    if (nv > 0) bp_gamma_kernel<<<grid_blocks(nv), 256, 0, st>>>(x0, x1, nv, sc);
    unsigned long long gb[3];
    if (cudaMemcpyAsync(gb, sc->gamma_bits, sizeof(gb), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return CCD_ERR_CUDA;
    const double K[2] = {30.0 * 0x1p-52, 28.0 * 0x1p-52};   // VF, EE
    for (int k = 0; k < 2; ++k)
        for (int c = 0; c < 3; ++c) {
            double g;
            memcpy(&g, &gb[c], sizeof(g));
            eps[3 * k + c] = K[k] * ((g * g) * g);
        }
    return CCD_OK;
}

double pow2_at_least(double x)
{
    double h = 1.0;
    if (!(x > 0.0)) return 0x1p-60;
    while (h < x) h *= 2.0;
    while (h * 0.5 >= x) h *= 0.5;
    return h;
}

}  // namespace

extern "C" {

ccd_status ccd_scene_eps(const double *x0, const double *x1, int64_t nv, double eps[6],
                         void *workspace, size_t ws_bytes, void *stream)
{
    if (!eps || nv < 0 || (nv > 0 && (!x0 || !x1))) return CCD_ERR_ARG;
    if (!workspace || ws_bytes < sizeof(BpScene)) return CCD_ERR_WORKSPACE;
    return scene_eps(x0, x1, nv, (BpScene *)workspace, eps, (cudaStream_t)stream);
}

size_t ccd_broad_phase_workspace_bytes(int64_t nv, int64_t nf, int64_t ne, int64_t cap_vf,
                                       int64_t cap_ee)
{
    if (nv < 0 || nf < 0 || ne < 0 || cap_vf < 0 || cap_ee < 0 ||
        BP_SLOTS * (nv + nf + ne) >= 0x7fffffffLL || cap_vf >= 0x7fffffffLL ||
        cap_ee >= 0x7fffffffLL)
        return 0;
    BpLayout L;
    return bp_layout(nv, nf, ne, cap_vf, cap_ee, &L) ? L.total : 0;
}

ccd_status ccd_broad_phase(const double *x0, const double *x1, int64_t nv, const int32_t *faces,
                           int64_t nf, const int32_t *edges, int64_t ne, double margin,
                           int32_t *vf_pairs, int64_t cap_vf, int32_t *ee_pairs, int64_t cap_ee,
                           int64_t counts[2], void *workspace, size_t ws_bytes, void *stream)
{
    if (!counts || nv < 0 || nf < 0 || ne < 0 || cap_vf < 0 || cap_ee < 0 || !(margin >= 0.0) ||
        BP_SLOTS * (nv + nf + ne) >= 0x7fffffffLL || (nv > 0 && (!x0 || !x1)) ||
        (nf > 0 && !faces) || (ne > 0 && !edges) || (cap_vf > 0 && !vf_pairs) ||
        (cap_ee > 0 && !ee_pairs) || nv >= (1LL << 31))
        return CCD_ERR_ARG;
    counts[0] = counts[1] = 0;
    BpLayout L;
    if (!bp_layout(nv, nf, ne, cap_vf, cap_ee, &L)) return CCD_ERR_CUDA;
    if (!workspace || ws_bytes < L.total) return CCD_ERR_WORKSPACE;
    const long long np = nv + nf + ne, m = BP_SLOTS * np;
    if (np == 0) return CCD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    BpScene *sc = (BpScene *)(ws + L.scene);
    double *boxes = (double *)(ws + L.boxes);
    bp_init_kernel<<<1, 32, 0, st>>>(sc);
    bp_boxes_kernel<<<grid_blocks(np), 256, 0, st>>>(x0, x1, nv, nf, ne, faces, edges, margin,
                                                     boxes, sc);
    BpScene host;
    if (cudaMemcpyAsync(&host, sc, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return CCD_ERR_CUDA;
    // the grid: cell edge a power of two >= 1.01 x the largest extent, at
    // most 2^20 cells per axis
    Grid g;
    double ext;
    {
        const unsigned long long b = host.ext_bits;
        memcpy(&ext, &b, sizeof(ext));
    }
    g.h = pow2_at_least(ext * 1.01);
    for (int c = 0; c < 3; ++c) {
        long long lk = host.lo_key[c], hk = host.hi_key[c];
        lk ^= (lk >> 63) & 0x7fffffffffffffffLL;
        hk ^= (hk >> 63) & 0x7fffffffffffffffLL;
        double lo, hi;
        memcpy(&lo, &lk, sizeof(lo));
        memcpy(&hi, &hk, sizeof(hi));
        g.o[c] = lo;
        while ((hi - lo) / g.h >= (double)(1 << 20)) g.h *= 2.0;
    }
    unsigned long long *k0 = (unsigned long long *)(ws + L.keys0);
    unsigned long long *k1 = (unsigned long long *)(ws + L.keys1);
    int *v0 = (int *)(ws + L.vals0), *v1 = (int *)(ws + L.vals1);
    bp_entries_kernel<<<grid_blocks(np), 256, 0, st>>>(boxes, np, g, k0, v0);
    size_t tb = L.temp_bytes;
    if (cub::DeviceRadixSort::SortPairs(ws + L.temp, tb, k0, k1, v0, v1, (int)m, 0, 64, st) !=
        cudaSuccess)
        return CCD_ERR_CUDA;
    unsigned long long *c0 = (unsigned long long *)(ws + L.cand0);
    unsigned long long *c1 = (unsigned long long *)(ws + L.cand1);
    // VF candidates into c0, EE candidates into c1 (each at most its cap)
    bp_pairs_kernel<<<grid_blocks(m), 256, 0, st>>>(k1, v1, m, boxes, nv, nf, faces, edges, g, c0,
                                                    cap_vf, c1, cap_ee, sc);
    if (cudaMemcpyAsync(&host, sc, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return CCD_ERR_CUDA;
    counts[0] = (int64_t)host.vf_count;
    counts[1] = (int64_t)host.ee_count;
    if (counts[0] > cap_vf || counts[1] > cap_ee) return CCD_ERR_CAPACITY;
    // deterministic order: sort each list by (first id, second id)
    for (int k = 0; k < 2; ++k) {
        const long long n = counts[k];
        if (n == 0) continue;
        unsigned long long *src = k == 0 ? c0 : c1;
        unsigned long long *dst = (unsigned long long *)(ws + L.cand2);
        tb = L.temp_bytes;
        if (cub::DeviceRadixSort::SortKeys(ws + L.temp, tb, src, dst, (int)n, 0, 64, st) !=
            cudaSuccess)
            return CCD_ERR_CUDA;
        bp_unpack_kernel<<<grid_blocks(n), 256, 0, st>>>(dst, n, k == 0 ? vf_pairs : ee_pairs);
    }
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}

size_t ccd_active_set_workspace_bytes(int64_t n_cand, int64_t max_itr)
{
    if (n_cand < 0 || n_cand >= 0x7fffffffLL) return 0;
    const size_t m = ccd_multi_workspace_bytes(n_cand, max_itr, nullptr);
    if (m == 0) return 0;
    size_t t = 0;
    if (cub::DeviceScan::ExclusiveSum(nullptr, t, (int *)nullptr, (int *)nullptr,
                                      (int)(n_cand > 0 ? n_cand : 1)) != cudaSuccess)
        return 0;
    const size_t n = (size_t)n_cand;
    return 1024 + al256(24 * sizeof(double) * n) + al256(n) + 2 * al256(sizeof(double) * n) +
           2 * al256(sizeof(int) * n) + al256(t) + m;
}

ccd_status ccd_active_set(const double *x0, const double *x1, int64_t nv, const int32_t *faces,
                          const int32_t *edges, const int32_t *vf_pairs, int64_t n_vf,
                          const int32_t *ee_pairs, int64_t n_ee, double delta, int64_t max_itr,
                          int32_t *out_kind, int32_t *out_pairs, double *out_toi,
                          int64_t *n_active, double eps_out[6], void *workspace, size_t ws_bytes,
                          void *stream)
{
    if (!n_active || n_vf < 0 || n_ee < 0 || nv < 0 || !(delta > 0.0) || max_itr < 1)
        return CCD_ERR_ARG;
    const long long n = n_vf + n_ee;
    if (n > 0 && (!x0 || !x1 || !out_kind || !out_pairs || !out_toi ||
                  (n_vf > 0 && (!faces || !vf_pairs)) || (n_ee > 0 && (!edges || !ee_pairs))))
        return CCD_ERR_ARG;
    const size_t need = ccd_active_set_workspace_bytes(n, max_itr);
    if (need == 0) return CCD_ERR_CUDA;
    if (!workspace || ws_bytes < need) return CCD_ERR_WORKSPACE;
    *n_active = 0;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    BpScene *sc = (BpScene *)ws;                       // gamma only
    ccd_segment *dsegs = (ccd_segment *)(ws + 256);    // 2 segments
    size_t off = 1024;
    double *soa = (double *)(ws + off); off += al256(24 * sizeof(double) * (size_t)n);
    uint8_t *collides = (uint8_t *)(ws + off); off += al256((size_t)n);
    double *toi = (double *)(ws + off); off += al256(sizeof(double) * (size_t)n);
    double *out_tol = (double *)(ws + off); off += al256(sizeof(double) * (size_t)n);
    int *flags = (int *)(ws + off); off += al256(sizeof(int) * (size_t)n);
    int *pos = (int *)(ws + off); off += al256(sizeof(int) * (size_t)n);
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, (int *)nullptr, (int *)nullptr,
                                  (int)(n > 0 ? n : 1));
    void *temp = ws + off; off += al256(tb);
    char *mws = ws + off;
    const size_t mws_bytes = ws_bytes - off;

    double eps[6];
    ccd_status r = scene_eps(x0, x1, nv, sc, eps, st);
    if (r != CCD_OK) return r;
    ccd_segment segs[2];
    for (int k = 0; k < 2; ++k) {
        segs[k].offset = k == 0 ? 0 : n_vf;
        segs[k].count = k == 0 ? n_vf : n_ee;
        segs[k].kind = k == 0 ? CCD_KIND_VF : CCD_KIND_EE;
        segs[k].group = 0;
        for (int c = 0; c < 3; ++c) {
            segs[k].err[c] = eps[3 * k + c];
            if (eps_out) eps_out[3 * k + c] = eps[3 * k + c];
        }
        segs[k].ms = 0.0;
        segs[k].delta = delta;
        segs[k].max_itr = max_itr;
        segs[k].t_max = 1.0;
    }
    if (n == 0) return CCD_OK;
    if (cudaMemcpyAsync(dsegs, segs, sizeof(segs), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return CCD_ERR_CUDA;
    as_gather_kernel<<<grid_blocks(n), 256, 0, st>>>(x0, x1, faces, edges, vf_pairs, n_vf,
                                                     ee_pairs, n_ee, soa);
    r = ccd_multi_batch(soa, n, dsegs, 2, max_itr, collides, toi, out_tol, nullptr, nullptr, mws,
                        mws_bytes, stream);
    if (r != CCD_OK) return r;
    // Algorithm 3: keep (c, t) when 0 <= t <= 1, i.e. a reported collision
    as_flags_kernel<<<grid_blocks(n), 256, 0, st>>>(collides, n, flags);
    if (cub::DeviceScan::ExclusiveSum(temp, tb, flags, pos, (int)n, st) != cudaSuccess)
        return CCD_ERR_CUDA;
    as_scatter_kernel<<<grid_blocks(n), 256, 0, st>>>(flags, pos, n, n_vf, vf_pairs, ee_pairs,
                                                      toi, out_kind, out_pairs, out_toi);
    int last_pos = 0, last_flag = 0;
    int32_t status = 0;
    if (cudaMemcpyAsync(&last_pos, pos + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&last_flag, flags + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        ccd_workspace_status(mws, &status, nullptr, stream) != CCD_OK)
        return CCD_ERR_CUDA;
    *n_active = (int64_t)last_pos + last_flag;
    return status == CCD_OK ? CCD_OK : (ccd_status)status;
}

}  // extern "C"
