// DAX and DAS compressed operation matrices on the device (Sec. III-A).
//
// DAX entry = (uint64 row-major index, complex value); DAS entry = (uint64
// distance word: zeros since the previous non-zero of the row, bit 63 = last
// of its row, complex value).  Both keep a derived row pointer (first entry
// of every row) so that the MTP and the MVM kernels can place and find rows
// without searching.  For DAS the row pointer is what parsing the distance
// words yields (a scan over the row-end flags); for DAX it comes from the
// sorted indices.
//
// MTP (Fig. 2): every pair (a, b) of entries gives one result entry.  With
// rows r_a, r_b, the result row r_a * dim_b + r_b starts at
//     rowptr_a[r_a] * nnz_b + nnz_row_a(r_a) * rowptr_b[r_b]
// and inside it the entries of a's row (outer) times b's row (inner) are in
// column order, so each thread writes its entry straight to its final
// position: the result is in row-major order with no sort.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

struct mera_dax {
    int nq = 0;
    uint64_t nnz = 0;
    unsigned long long* idx = nullptr;   // row-major linear index
    double2* val = nullptr;
    unsigned long long* rowptr = nullptr;  // 2^nq + 1
};

struct mera_das {
    int nq = 0;
    uint64_t nnz = 0;
    unsigned long long* dist = nullptr;  // zeros before | bit 63 = last of row
    double2* val = nullptr;
    unsigned long long* rowptr = nullptr;  // 2^nq + 1, from the row-end flags
    unsigned long long* tail = nullptr;    // zeros after the last non-zero, per row
};

namespace mera {

static constexpr unsigned long long LAST = 1ull << 63;
static constexpr unsigned long long DMASK = LAST - 1ull;

static int grid64(uint64_t work, int threads) {
    uint64_t b = (work + threads - 1) / threads;
    if (b > 152ull * 64) b = 152ull * 64;
    if (b < 1) b = 1;
    return (int)b;
}

// ------------------------------------------------------------- kernels ----
// rowptr[r] = first entry with index >= r * dim (binary search; r = 0..dim)
__global__ void k_dax_rowptr(const unsigned long long* __restrict__ idx, uint64_t nnz, int nq,
                             unsigned long long* __restrict__ rowptr) {
    const uint64_t dim = 1ull << nq;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= dim; r += stride) {
        const unsigned long long key = r << nq;   // r = dim, nq = 32 wraps to 0: handled below
        uint64_t lo = 0, hi = nnz;
        if (r == dim) {
            lo = nnz;
        } else {
            while (lo < hi) {
                const uint64_t mid = (lo + hi) >> 1;
                if (idx[mid] < key) lo = mid + 1;
                else hi = mid;
            }
        }
        rowptr[r] = lo;
    }
}

// Row pointer of a (x) b, directly from the factors' row pointers.
__global__ void k_kron_rowptr(const unsigned long long* __restrict__ ra, const unsigned long long* __restrict__ rb,
                              int nqb, uint64_t nnzb, uint64_t nnzc, uint64_t dimc,
                              unsigned long long* __restrict__ rc) {
    const uint64_t dimb = 1ull << nqb;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= dimc; r += stride) {
        if (r == dimc) {
            rc[r] = nnzc;
            continue;
        }
        const uint64_t a = r >> nqb, b = r & (dimb - 1);
        rc[r] = ra[a] * nnzb + (ra[a + 1] - ra[a]) * rb[b];
    }
}

// Largest r with rowptr[r] <= p (the row holding entry p).
__device__ __forceinline__ uint64_t row_of(const unsigned long long* rowptr, uint64_t dim, uint64_t p) {
    uint64_t lo = 0, hi = dim;   // rowptr[lo] <= p < rowptr[hi]
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (rowptr[mid] <= p) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}

// DAX MTP: thread per entry pair (ia outer, ib inner).
__global__ void k_dax_kron(const mera_dax A, const mera_dax B, unsigned long long* __restrict__ idxc,
                           double2* __restrict__ valc) {
    const uint64_t total = A.nnz * B.nnz;
    const int nqc = A.nq + B.nq;
    const uint64_t dimb = 1ull << B.nq, dima = 1ull << A.nq;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint64_t ia = t / B.nnz, ib = t - ia * B.nnz;
        const unsigned long long xa = A.idx[ia], xb = B.idx[ib];
        const uint64_t ra = xa >> A.nq, ca = xa & (dima - 1);
        const uint64_t rb = xb >> B.nq, cb = xb & (dimb - 1);
        const uint64_t a0 = A.rowptr[ra], na = A.rowptr[ra + 1] - a0;
        const uint64_t b0 = B.rowptr[rb], nb = B.rowptr[rb + 1] - b0;
        const uint64_t p = a0 * B.nnz + na * b0 + (ia - a0) * nb + (ib - b0);
        const uint64_t row = ra * dimb + rb, col = ca * dimb + cb;
        idxc[p] = (nqc >= 64 ? 0ull : (row << nqc)) | col;
        valc[p] = cmul_d(A.val[ia], B.val[ib]);
    }
}

// DAS MTP: the three-case distance equation of Sec. III-A.2.
__global__ void k_das_kron(const mera_das A, const mera_das B, unsigned long long* __restrict__ distc,
                           double2* __restrict__ valc) {
    const uint64_t total = A.nnz * B.nnz;
    const uint64_t dima = 1ull << A.nq, dimb = 1ull << B.nq;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint64_t ia = t / B.nnz, ib = t - ia * B.nnz;
        const uint64_t ra = row_of(A.rowptr, dima, ia), rb = row_of(B.rowptr, dimb, ib);
        const uint64_t a0 = A.rowptr[ra], na = A.rowptr[ra + 1] - a0;
        const uint64_t b0 = B.rowptr[rb], nb = B.rowptr[rb + 1] - b0;
        const unsigned long long wa = A.dist[ia], wb = B.dist[ib];
        const uint64_t adis = wa & DMASK, bdis = wb & DMASK;
        uint64_t dis;
        if (ia == a0 && ib == b0) dis = adis * dimb + bdis;                 // case 1
        else if (ib == b0) dis = adis * dimb + bdis + B.tail[rb];           // case 2
        else dis = bdis;                                                    // otherwise
        const bool last = (wa & LAST) && (wb & LAST);
        const uint64_t p = a0 * B.nnz + na * b0 + (ia - a0) * nb + (ib - b0);
        distc[p] = dis | (last ? LAST : 0ull);
        valc[p] = cmul_d(A.val[ia], B.val[ib]);
    }
}

// DAS parse, step 1: row-end flags per block (blocks of 1024 entries).
__global__ void k_das_count(const unsigned long long* __restrict__ dist, uint64_t nnz,
                            unsigned long long* __restrict__ bcount) {
    __shared__ unsigned int sh[32];
    const uint64_t base = (uint64_t)blockIdx.x * 1024;
    unsigned int c = 0;
    for (int j = threadIdx.x; j < 1024; j += blockDim.x) {
        const uint64_t p = base + j;
        if (p < nnz && (dist[p] & LAST)) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        bcount[blockIdx.x] = s;
    }
}

// Step 2: exclusive scan of the block counts (one block, sequential chunks).
__global__ void k_scan_single(unsigned long long* __restrict__ v, uint64_t n) {
    __shared__ unsigned long long part[1024];
    const uint64_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint64_t lo = threadIdx.x * per, hi = min(n, lo + per);
    unsigned long long s = 0;
    for (uint64_t i = lo; i < hi; ++i) s += v[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int j = 0; j < (int)blockDim.x; ++j) {
            const unsigned long long x = part[j];
            part[j] = run;
            run += x;
        }
    }
    __syncthreads();
    unsigned long long run = part[threadIdx.x];
    for (uint64_t i = lo; i < hi; ++i) {
        const unsigned long long x = v[i];
        v[i] = run;
        run += x;
    }
}

// Step 3: every row-end entry p of row r writes rowptr[r + 1] = p + 1.
__global__ void k_das_rowptr(const unsigned long long* __restrict__ dist, uint64_t nnz,
                             const unsigned long long* __restrict__ boff, unsigned long long* __restrict__ rowptr) {
    __shared__ unsigned int warp_tot[32];
    const uint64_t base = (uint64_t)blockIdx.x * 1024;
    // each thread owns 1024 / blockDim.x consecutive entries
    const int per = 1024 / blockDim.x;
    const uint64_t p0 = base + (uint64_t)threadIdx.x * per;
    unsigned int c = 0;
    for (int j = 0; j < per; ++j)
        if (p0 + j < nnz && (dist[p0 + j] & LAST)) ++c;
    // block exclusive scan of c
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int run = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            const unsigned int x = warp_tot[k];
            warp_tot[k] = run;
            run += x;
        }
    }
    __syncthreads();
    unsigned long long r = boff[blockIdx.x] + warp_tot[w] + (incl - c);
    for (int j = 0; j < per; ++j) {
        const uint64_t p = p0 + j;
        if (p < nnz && (dist[p] & LAST)) rowptr[++r] = p + 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rowptr[0] = 0;
}

// Trailing zeros of every row: dim - 1 - (last column).
__global__ void k_das_tail(const unsigned long long* __restrict__ dist, const unsigned long long* __restrict__ rowptr,
                           int nq, unsigned long long* __restrict__ tail) {
    const uint64_t dim = 1ull << nq;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += stride) {
        uint64_t col = ~0ull;   // -1: the column before the row start
        for (uint64_t p = rowptr[r]; p < rowptr[r + 1]; ++p) col += (dist[p] & DMASK) + 1;
        tail[r] = dim - 1 - col;
    }
}

template <typename V>
__device__ __forceinline__ V from_d(double2 v);
template <>
__device__ __forceinline__ double2 from_d<double2>(double2 v) {
    return v;
}
template <>
__device__ __forceinline__ float2 from_d<float2>(double2 v) {
    return make_float2((float)v.x, (float)v.y);
}

// DAX MVM: out[r] = sum over the row's entries of value * in[col].
template <typename V>
__global__ void k_dax_mvm(const mera_dax D, const V* __restrict__ in, V* __restrict__ out) {
    const uint64_t dim = 1ull << D.nq;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += stride) {
        V acc;
        acc.x = 0;
        acc.y = 0;
        for (uint64_t p = D.rowptr[r]; p < D.rowptr[r + 1]; ++p)
            acc = cfma(from_d<V>(D.val[p]), in[D.idx[p] & (dim - 1)], acc);
        out[r] = acc;
    }
}

// DAS MVM: the column is parsed from the distance words along the row.
template <typename V>
__global__ void k_das_mvm(const mera_das D, const V* __restrict__ in, V* __restrict__ out) {
    const uint64_t dim = 1ull << D.nq;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += stride) {
        V acc;
        acc.x = 0;
        acc.y = 0;
        uint64_t col = ~0ull;
        for (uint64_t p = D.rowptr[r]; p < D.rowptr[r + 1]; ++p) {
            col += (D.dist[p] & DMASK) + 1;
            acc = cfma(from_d<V>(D.val[p]), in[col], acc);
        }
        out[r] = acc;
    }
}

// ------------------------------------------------------------ host side ---
template <typename T>
static int dalloc(T** p, uint64_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%llu bytes): %s", (unsigned long long)(count * sizeof(T)), cudaGetErrorString(e));
        return MERA_ENOMEM;
    }
    return MERA_OK;
}

static void free_dax(mera_dax* d) {
    if (!d) return;
    cudaFree(d->idx);
    cudaFree(d->val);
    cudaFree(d->rowptr);
    delete d;
}
static void free_das(mera_das* d) {
    if (!d) return;
    cudaFree(d->dist);
    cudaFree(d->val);
    cudaFree(d->rowptr);
    cudaFree(d->tail);
    delete d;
}

static int dax_alloc(int nq, uint64_t nnz, mera_dax** out) {
    mera_dax* d = new mera_dax();
    d->nq = nq;
    d->nnz = nnz;
    int st = dalloc(&d->idx, nnz);
    if (st == MERA_OK) st = dalloc(&d->val, nnz);
    if (st == MERA_OK) st = dalloc(&d->rowptr, (1ull << nq) + 1);
    if (st != MERA_OK) {
        free_dax(d);
        return st;
    }
    *out = d;
    return MERA_OK;
}

static int das_alloc(int nq, uint64_t nnz, mera_das** out) {
    mera_das* d = new mera_das();
    d->nq = nq;
    d->nnz = nnz;
    int st = dalloc(&d->dist, nnz);
    if (st == MERA_OK) st = dalloc(&d->val, nnz);
    if (st == MERA_OK) st = dalloc(&d->rowptr, (1ull << nq) + 1);
    if (st == MERA_OK) st = dalloc(&d->tail, 1ull << nq);
    if (st != MERA_OK) {
        free_das(d);
        return st;
    }
    *out = d;
    return MERA_OK;
}

static int dax_finish(mera_dax* d, cudaStream_t st) {
    const uint64_t dim = 1ull << d->nq;
    launch_begin(st, MERA_KCLASS_DAX, 8.0 * (dim + 1));
    k_dax_rowptr<<<grid64(dim + 1, 256), 256, 0, st>>>(d->idx, d->nnz, d->nq, d->rowptr);
    return launch_end(st);
}

static int das_finish(mera_das* d, cudaStream_t st) {
    const uint64_t dim = 1ull << d->nq;
    const uint64_t nb = (d->nnz + 1023) / 1024;
    unsigned long long* boff = nullptr;
    MERA_TRY(dalloc(&boff, nb));
    int rc = MERA_OK;
    launch_begin(st, MERA_KCLASS_DAX, 8.0 * d->nnz);
    k_das_count<<<(unsigned)nb, 256, 0, st>>>(d->dist, d->nnz, boff);
    rc = launch_end(st);
    if (rc == MERA_OK) {
        launch_begin(st, MERA_KCLASS_DAX, 16.0 * nb);
        k_scan_single<<<1, 1024, 0, st>>>(boff, nb);
        rc = launch_end(st);
    }
    if (rc == MERA_OK) {
        launch_begin(st, MERA_KCLASS_DAX, 8.0 * d->nnz + 8.0 * dim);
        k_das_rowptr<<<(unsigned)nb, 256, 0, st>>>(d->dist, d->nnz, boff, d->rowptr);
        rc = launch_end(st);
    }
    if (rc == MERA_OK) {
        launch_begin(st, MERA_KCLASS_DAX, 8.0 * d->nnz + 16.0 * dim);
        k_das_tail<<<grid64(dim, 256), 256, 0, st>>>(d->dist, d->rowptr, d->nq, d->tail);
        rc = launch_end(st);
    }
    cudaStreamSynchronize(st);   // boff is freed right after
    cudaFree(boff);
    return rc;
}

static int check_nq(int nq) {
    MERA_RETURN_IF(nq < 0 || nq > 32, MERA_EINVAL, "nq=%d outside [0, 32]", nq);
    return MERA_OK;
}

}  // namespace mera

using namespace mera;

#define API_TRY try {
#define API_CATCH                                  \
    }                                              \
    catch (const std::bad_alloc&) {                \
        set_error("host allocation failed");       \
        return MERA_ENOMEM;                        \
    }                                              \
    catch (...) {                                  \
        set_error("unexpected C++ exception");     \
        return MERA_EINVAL;                        \
    }

extern "C" {

int mera_dax_from_host(int nq, uint64_t nnz, const uint64_t* index, const double* vals, void* stream,
                       mera_dax** out) {
    API_TRY
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    *out = nullptr;
    MERA_TRY(check_nq(nq));
    MERA_RETURN_IF(nnz > 0 && (index == nullptr || vals == nullptr), MERA_EINVAL, "NULL array");
    const unsigned __int128 cells = (unsigned __int128)1 << (2 * nq);
    for (uint64_t p = 0; p < nnz; ++p) {
        MERA_RETURN_IF((unsigned __int128)index[p] >= cells, MERA_EINVAL, "index %llu out of range",
                       (unsigned long long)index[p]);
        MERA_RETURN_IF(p > 0 && index[p] <= index[p - 1], MERA_EINVAL, "indices must ascend (entry %llu)",
                       (unsigned long long)p);
    }
    cudaStream_t st = (cudaStream_t)stream;
    mera_dax* d = nullptr;
    MERA_TRY(dax_alloc(nq, nnz, &d));
    cudaError_t e = cudaMemcpyAsync(d->idx, index, nnz * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d->val, vals, nnz * 16, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        free_dax(d);
        set_error("upload: %s", cudaGetErrorString(e));
        return MERA_ECUDA;
    }
    int rc = dax_finish(d, st);
    if (rc == MERA_OK) rc = cudaStreamSynchronize(st) == cudaSuccess ? MERA_OK : MERA_ECUDA;
    if (rc != MERA_OK) {
        free_dax(d);
        return rc;
    }
    *out = d;
    return MERA_OK;
    API_CATCH
}

int mera_das_from_host(int nq, uint64_t nnz, const uint64_t* dist, const double* vals, void* stream,
                       mera_das** out) {
    API_TRY
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    *out = nullptr;
    MERA_TRY(check_nq(nq));
    MERA_RETURN_IF(nnz > 0 && (dist == nullptr || vals == nullptr), MERA_EINVAL, "NULL array");
    // validate the row structure: dim rows, each ending with a flagged entry,
    // columns inside the row
    const uint64_t dim = 1ull << nq;
    uint64_t rows = 0;
    unsigned long long col = ~0ull;
    for (uint64_t p = 0; p < nnz; ++p) {
        col += (dist[p] & DMASK) + 1;
        MERA_RETURN_IF(col >= dim, MERA_EINVAL, "entry %llu: column beyond the row", (unsigned long long)p);
        if (dist[p] & LAST) {
            ++rows;
            col = ~0ull;
        }
    }
    MERA_RETURN_IF(rows != dim || (nnz > 0 && !(dist[nnz - 1] & LAST)), MERA_EINVAL,
                   "DAS needs %llu rows each ending with a flagged entry", (unsigned long long)dim);
    cudaStream_t st = (cudaStream_t)stream;
    mera_das* d = nullptr;
    MERA_TRY(das_alloc(nq, nnz, &d));
    cudaError_t e = cudaMemcpyAsync(d->dist, dist, nnz * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d->val, vals, nnz * 16, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        free_das(d);
        set_error("upload: %s", cudaGetErrorString(e));
        return MERA_ECUDA;
    }
    int rc = das_finish(d, st);
    if (rc != MERA_OK) {
        free_das(d);
        return rc;
    }
    *out = d;
    return MERA_OK;
    API_CATCH
}

int mera_dax_from_dense(const double* m, int nq, void* stream, mera_dax** out) {
    API_TRY
    MERA_RETURN_IF(m == nullptr || out == nullptr, MERA_EINVAL, "NULL argument");
    MERA_RETURN_IF(nq < 0 || nq > 12, MERA_EINVAL, "dense input limited to nq <= 12");
    const uint64_t dim = 1ull << nq;
    std::vector<uint64_t> idx;
    std::vector<double> val;
    for (uint64_t r = 0; r < dim; ++r)
        for (uint64_t c = 0; c < dim; ++c) {
            const double re = m[2 * (r * dim + c)], im = m[2 * (r * dim + c) + 1];
            if (re != 0.0 || im != 0.0) {
                idx.push_back(r * dim + c);
                val.push_back(re);
                val.push_back(im);
            }
        }
    return mera_dax_from_host(nq, idx.size(), idx.data(), val.data(), stream, out);
    API_CATCH
}

int mera_das_from_dense(const double* m, int nq, void* stream, mera_das** out) {
    API_TRY
    MERA_RETURN_IF(m == nullptr || out == nullptr, MERA_EINVAL, "NULL argument");
    MERA_RETURN_IF(nq < 0 || nq > 12, MERA_EINVAL, "dense input limited to nq <= 12");
    const uint64_t dim = 1ull << nq;
    std::vector<uint64_t> dist;
    std::vector<double> val;
    for (uint64_t r = 0; r < dim; ++r) {
        long long prev = -1;
        size_t first = dist.size();
        for (uint64_t c = 0; c < dim; ++c) {
            const double re = m[2 * (r * dim + c)], im = m[2 * (r * dim + c) + 1];
            if (re != 0.0 || im != 0.0) {
                dist.push_back((uint64_t)((long long)c - prev - 1));
                val.push_back(re);
                val.push_back(im);
                prev = (long long)c;
            }
        }
        MERA_RETURN_IF(dist.size() == first, MERA_EINVAL, "row %llu has no non-zero", (unsigned long long)r);
        dist.back() |= LAST;
    }
    return mera_das_from_host(nq, dist.size(), dist.data(), val.data(), stream, out);
    API_CATCH
}

int mera_dax_kron(const mera_dax* a, const mera_dax* b, void* stream, mera_dax** out) {
    API_TRY
    MERA_RETURN_IF(a == nullptr || b == nullptr || out == nullptr, MERA_EINVAL, "NULL argument");
    *out = nullptr;
    MERA_TRY(check_nq(a->nq + b->nq));
    const uint64_t nnz = a->nnz * b->nnz;
    MERA_RETURN_IF(a->nnz != 0 && nnz / a->nnz != b->nnz, MERA_EINVAL, "entry count overflows");
    cudaStream_t st = (cudaStream_t)stream;
    mera_dax* c = nullptr;
    MERA_TRY(dax_alloc(a->nq + b->nq, nnz, &c));
    const uint64_t dimc = 1ull << c->nq;
    launch_begin(st, MERA_KCLASS_DAX, 8.0 * (dimc + 1));
    k_kron_rowptr<<<grid64(dimc + 1, 256), 256, 0, st>>>(a->rowptr, b->rowptr, b->nq, b->nnz, nnz, dimc, c->rowptr);
    int rc = launch_end(st);
    if (rc == MERA_OK && nnz > 0) {
        launch_begin(st, MERA_KCLASS_DAX, 24.0 * (double)nnz + 24.0 * (double)(a->nnz + b->nnz));
        k_dax_kron<<<grid64(nnz, 256), 256, 0, st>>>(*a, *b, c->idx, c->val);
        rc = launch_end(st);
    }
    if (rc != MERA_OK) {
        free_dax(c);
        return rc;
    }
    *out = c;
    return MERA_OK;
    API_CATCH
}

int mera_das_kron(const mera_das* a, const mera_das* b, void* stream, mera_das** out) {
    API_TRY
    MERA_RETURN_IF(a == nullptr || b == nullptr || out == nullptr, MERA_EINVAL, "NULL argument");
    *out = nullptr;
    MERA_TRY(check_nq(a->nq + b->nq));
    const uint64_t nnz = a->nnz * b->nnz;
    MERA_RETURN_IF(a->nnz != 0 && nnz / a->nnz != b->nnz, MERA_EINVAL, "entry count overflows");
    cudaStream_t st = (cudaStream_t)stream;
    mera_das* c = nullptr;
    MERA_TRY(das_alloc(a->nq + b->nq, nnz, &c));
    const uint64_t dimc = 1ull << c->nq;
    launch_begin(st, MERA_KCLASS_DAX, 8.0 * (dimc + 1));
    k_kron_rowptr<<<grid64(dimc + 1, 256), 256, 0, st>>>(a->rowptr, b->rowptr, b->nq, b->nnz, nnz, dimc, c->rowptr);
    int rc = launch_end(st);
    if (rc == MERA_OK && nnz > 0) {
        launch_begin(st, MERA_KCLASS_DAX, 24.0 * (double)nnz + 24.0 * (double)(a->nnz + b->nnz));
        k_das_kron<<<grid64(nnz, 256), 256, 0, st>>>(*a, *b, c->dist, c->val);
        rc = launch_end(st);
    }
    if (rc == MERA_OK) {
        launch_begin(st, MERA_KCLASS_DAX, 8.0 * (double)nnz + 16.0 * dimc);
        k_das_tail<<<grid64(dimc, 256), 256, 0, st>>>(c->dist, c->rowptr, c->nq, c->tail);
        rc = launch_end(st);
    }
    if (rc != MERA_OK) {
        free_das(c);
        return rc;
    }
    *out = c;
    return MERA_OK;
    API_CATCH
}

static int mvm_check(int nq, mera_state* in, mera_state* out) {
    MERA_RETURN_IF(in == nullptr || out == nullptr, MERA_EINVAL, "NULL state");
    MERA_RETURN_IF(in->n != nq || out->n != nq, MERA_EINVAL, "states must have n = nq = %d", nq);
    MERA_RETURN_IF(in->dtype != out->dtype, MERA_EINVAL, "states must share the dtype");
    MERA_RETURN_IF(in->data == out->data, MERA_EINVAL, "the MVM is out of place: in and out must differ");
    return MERA_OK;
}

// Order out's stream after in's queued work.
static int join_streams(mera_state* in, mera_state* out) {
    if (in->stream == out->stream) return MERA_OK;
    cudaEvent_t ev;
    MERA_CHECK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, in->stream);
    cudaStreamWaitEvent(out->stream, ev, 0);
    cudaEventDestroy(ev);
    return MERA_OK;
}

int mera_dax_mvm(const mera_dax* d, mera_state* in, mera_state* out) {
    API_TRY
    MERA_RETURN_IF(d == nullptr, MERA_EINVAL, "dax is NULL");
    MERA_TRY(mvm_check(d->nq, in, out));
    MERA_TRY(join_streams(in, out));
    const uint64_t dim = 1ull << d->nq;
    const size_t eb = elem_bytes(in->dtype);
    launch_begin(out->stream, MERA_KCLASS_DAX, 24.0 * d->nnz + (double)dim * (2.0 * eb + 8.0));
    if (in->dtype == MERA_C128)
        k_dax_mvm<double2><<<grid64(dim, 256), 256, 0, out->stream>>>(*d, (const double2*)in->data, (double2*)out->data);
    else
        k_dax_mvm<float2><<<grid64(dim, 256), 256, 0, out->stream>>>(*d, (const float2*)in->data, (float2*)out->data);
    return launch_end(out->stream);
    API_CATCH
}

int mera_das_mvm(const mera_das* d, mera_state* in, mera_state* out) {
    API_TRY
    MERA_RETURN_IF(d == nullptr, MERA_EINVAL, "das is NULL");
    MERA_TRY(mvm_check(d->nq, in, out));
    MERA_TRY(join_streams(in, out));
    const uint64_t dim = 1ull << d->nq;
    const size_t eb = elem_bytes(in->dtype);
    launch_begin(out->stream, MERA_KCLASS_DAX, 24.0 * d->nnz + (double)dim * (2.0 * eb + 8.0));
    if (in->dtype == MERA_C128)
        k_das_mvm<double2><<<grid64(dim, 256), 256, 0, out->stream>>>(*d, (const double2*)in->data, (double2*)out->data);
    else
        k_das_mvm<float2><<<grid64(dim, 256), 256, 0, out->stream>>>(*d, (const float2*)in->data, (float2*)out->data);
    return launch_end(out->stream);
    API_CATCH
}

int mera_dax_info(const mera_dax* d, int* nq, uint64_t* nnz) {
    MERA_RETURN_IF(d == nullptr, MERA_EINVAL, "dax is NULL");
    if (nq) *nq = d->nq;
    if (nnz) *nnz = d->nnz;
    return MERA_OK;
}

int mera_das_info(const mera_das* d, int* nq, uint64_t* nnz) {
    MERA_RETURN_IF(d == nullptr, MERA_EINVAL, "das is NULL");
    if (nq) *nq = d->nq;
    if (nnz) *nnz = d->nnz;
    return MERA_OK;
}

int mera_dax_export(const mera_dax* d, uint64_t* index, double* vals) {
    MERA_RETURN_IF(d == nullptr, MERA_EINVAL, "dax is NULL");
    MERA_CHECK_CUDA(cudaDeviceSynchronize());
    if (index) MERA_CHECK_CUDA(cudaMemcpy(index, d->idx, d->nnz * 8, cudaMemcpyDeviceToHost));
    if (vals) MERA_CHECK_CUDA(cudaMemcpy(vals, d->val, d->nnz * 16, cudaMemcpyDeviceToHost));
    return MERA_OK;
}

int mera_das_export(const mera_das* d, uint64_t* dist, double* vals) {
    MERA_RETURN_IF(d == nullptr, MERA_EINVAL, "das is NULL");
    MERA_CHECK_CUDA(cudaDeviceSynchronize());
    if (dist) MERA_CHECK_CUDA(cudaMemcpy(dist, d->dist, d->nnz * 8, cudaMemcpyDeviceToHost));
    if (vals) MERA_CHECK_CUDA(cudaMemcpy(vals, d->val, d->nnz * 16, cudaMemcpyDeviceToHost));
    return MERA_OK;
}

int mera_dax_destroy(mera_dax* d) {
    if (d) {
        cudaDeviceSynchronize();
        free_dax(d);
    }
    return MERA_OK;
}

int mera_das_destroy(mera_das* d) {
    if (d) {
        cudaDeviceSynchronize();
        free_das(d);
    }
    return MERA_OK;
}

}  // extern "C"
