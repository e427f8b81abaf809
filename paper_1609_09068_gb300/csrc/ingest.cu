// ingest.cu -- graph model of Sec. 3 and Def. 3.4: validate the CSR (simple
// digraph: sorted, duplicate-free rows), drop self-loops (Sec. 4.1 and 5.2
// ignore them), out-degree without loops, and the in-adjacency (CSC) with
// sources ascending inside each column (stable radix sort by target).
#include "common.cuh"
#include "spmv.cuh"

namespace prgb {

// The checks and the copy walk the entries, not the rows: a warp takes 1,024
// consecutive entries (lane l the entries base + l + 32 k), so every load of
// col and every store of the copy is one coalesced access whatever the row
// lengths, and a hub row is spread over many warps.  Each lane finds the row
// of its first entry by a binary search of rowptr and then steps forward.
constexpr int kWarpEntries = 1024;

// the row of entry e: rowptr[r] <= e < rowptr[r + 1] (rowptr checked first)
__device__ __forceinline__ int row_of(const int32_t* __restrict__ rowptr, int32_t n, int64_t e) {
  int lo = 0, hi = n;  // the answer is in [lo, hi)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)rowptr[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

// the offsets: non-decreasing, starting at 0 and ending at nnz
__global__ void validate_ptr_k(const int32_t* __restrict__ rowptr, int32_t n, int64_t nnz, uint8_t* has_loop,
                               Ctl* ctl) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rowptr[i], e = rowptr[i + 1];
    if ((s > e) || (s < 0) || (e > nnz) || (i == 0 && s != 0) || (i == n - 1 && e != nnz)) set_err(ctl, PR_EINVAL, 1);
    has_loop[i] = 0;
  }
}

// the entries: in range, strictly ascending within a row; a self-loop marks
// its row (at most one per row in a valid row)
__global__ void validate_cols_k(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t n,
                                int64_t nnz, uint8_t* has_loop, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (vload(&ctl->err)) return;  // bad offsets: the rows are not searchable
  for (int64_t base = gw * kWarpEntries; base < nnz; base += nw * kWarpEntries) {
    int64_t e = base + lane;
    if (e >= nnz) continue;
    int r = row_of(rowptr, n, e);
    bool bad = false;
    for (int k = 0; k < kWarpEntries / 32 && e < nnz; k++, e += 32) {
      while (r < n - 1 && (int64_t)rowptr[r + 1] <= e) r++;
      const int32_t c = col[e];
      if (c < 0 || c >= n) bad = true;
      if (e > rowptr[r] && col[e - 1] >= c) bad = true;
      if (c == r) has_loop[r] = 1;
    }
    if (bad) set_err(ctl, PR_EINVAL, 1);
  }
}

// loop-free out-degree of every row
__global__ void outdeg_k(const int32_t* __restrict__ rowptr, int32_t n, const uint8_t* __restrict__ has_loop,
                         int32_t* __restrict__ outdeg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    outdeg[i] = rowptr[i + 1] - rowptr[i] - (int32_t)has_loop[i];
}

// copy the non-loop entries and record the source row of every kept edge:
// entry e of row r goes to optr[r] + (e - rowptr[r]), one less when it
// follows the row's self-loop
__global__ void strip_loops_k(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t n,
                              int64_t nnz, const uint8_t* __restrict__ has_loop,
                              const int32_t* __restrict__ optr, int32_t* __restrict__ oidx,
                              uint32_t* __restrict__ key_dst, uint32_t* __restrict__ val_src) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = gw * kWarpEntries; base < nnz; base += nw * kWarpEntries) {
    int64_t e = base + lane;
    if (e >= nnz) continue;
    int r = row_of(rowptr, n, e);
    for (int k = 0; k < kWarpEntries / 32 && e < nnz; k++, e += 32) {
      while (r < n - 1 && (int64_t)rowptr[r + 1] <= e) r++;
      const int32_t c = col[e];
      if (c == r) continue;
      const int64_t pos = optr[r] + (e - rowptr[r]) - ((has_loop[r] && c > r) ? 1 : 0);
      oidx[pos] = c;
      key_dst[pos] = (uint32_t)c;
      val_src[pos] = (uint32_t)r;
    }
  }
}

// Column offsets from the edges' targets sorted ascending: iptr[x] = the
// number of edges whose target is below x, for x in [0, n].
__global__ void col_ptr_k(int64_t m, const uint32_t* __restrict__ tgt, int32_t n, int32_t* __restrict__ iptr) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = i == 0 ? 0 : (int64_t)tgt[i - 1] + 1;  // first column whose offset is i
    const int64_t hi = i == m ? (int64_t)n : (int64_t)tgt[i];  // last such column
    for (int64_t x = lo; x <= hi; x++) iptr[x] = (int32_t)i;
  }
}

// ---- PR_CANONICALIZE: sort every row and drop repeated columns -------------
// row offsets and column range are checked as in validate_rows_k (those are
// not fixable); each edge is tagged with its row
__global__ void edge_rows_k(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t n,
                            int64_t nnz, uint32_t* __restrict__ ecol, uint32_t* __restrict__ erow, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const int64_t s = rowptr[i], e = rowptr[i + 1];
    bool bad = (s > e) || (s < 0) || (e > nnz) || (i == 0 && s != 0) || (i == n - 1 && e != nnz);
    if (!bad) {
      for (int64_t k = s + lane; k < e; k += 32) {
        const int32_t c = col[k];
        if (c < 0 || c >= n) bad = true;
        ecol[k] = (uint32_t)c;
        erow[k] = (uint32_t)i;
      }
    }
    bad = __any_sync(0xffffffffu, bad);
    if (bad && lane == 0) set_err(ctl, PR_EINVAL, 2);
  }
}

// after the sort by (row, col): keep the first of each run of equal pairs
__global__ void dedup_flags_k(int64_t nnz, const uint32_t* __restrict__ erow, const uint32_t* __restrict__ ecol,
                              uint8_t* keepf, int32_t* rcnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
    const bool k = i == 0 || erow[i] != erow[i - 1] || ecol[i] != ecol[i - 1];
    keepf[i] = k;
    if (k) atomicAdd(&rcnt[erow[i]], 1);
  }
}

__global__ void dedup_compact_k(int64_t nnz, const uint32_t* __restrict__ ecol, const uint8_t* __restrict__ keepf,
                                const int32_t* __restrict__ kidx, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
    if (keepf[i]) out[kidx[i]] = (int32_t)ecol[i];
}

static unsigned grid_rows(int64_t n);

// rowptr / col (device) -> a CSR with sorted, duplicate-free rows in tmp
static pr_status canonicalize(const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz, Arena& tmp,
                              Ctl* ctl, int32_t** rp_out, int32_t** col_out, int64_t* nnz_out) {
  cudaStream_t s = tmp.stream();
  uint32_t *ecol, *erow, *kt, *vt;
  const size_t m1 = (size_t)(nnz > 0 ? nnz : 1);
  PRGB_TRY(tmp.alloc(&ecol, m1));
  PRGB_TRY(tmp.alloc(&erow, m1));
  PRGB_TRY(tmp.alloc(&kt, m1));
  PRGB_TRY(tmp.alloc(&vt, m1));
  if (n > 0) {
    edge_rows_k<<<grid_rows(n), kBlock, 0, s>>>(rowptr, col, n, nnz, ecol, erow, ctl);
    PRGB_LAUNCH();
  }
  int err = 0;
  PRGB_CUDA(cudaMemcpyAsync(&err, &ctl->err, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  if (err) return (pr_status)err;
  const int bits = bits_for((uint32_t)(n > 0 ? n - 1 : 0));
  // stable sorts: by column, then by row -> ordered by (row, column)
  PRGB_TRY(radix_sort_pairs(ecol, erow, kt, vt, nnz, bits, tmp));
  PRGB_TRY(radix_sort_pairs(erow, ecol, kt, vt, nnz, bits, tmp));
  uint8_t* keepf;
  int32_t *rcnt, *kidx, *rp, *cl;
  PRGB_TRY(tmp.alloc(&keepf, m1));
  PRGB_TRY(tmp.alloc(&rcnt, (size_t)n + 1));
  PRGB_TRY(tmp.alloc(&kidx, m1 + 1));
  PRGB_TRY(tmp.alloc(&rp, (size_t)n + 1));
  PRGB_CUDA(cudaMemsetAsync(rcnt, 0, ((size_t)n + 1) * 4, s));
  if (nnz > 0) {
    dedup_flags_k<<<grid_rows((nnz + 7) / 8), kBlock, 0, s>>>(nnz, erow, ecol, keepf, rcnt);
    PRGB_LAUNCH();
  }
  PRGB_TRY(scan_u8(keepf, kidx, nnz, tmp));
  PRGB_TRY(scan_i32(rcnt, rp, n, tmp));
  int32_t kept = 0;
  PRGB_CUDA(cudaMemcpyAsync(&kept, kidx + nnz, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  PRGB_TRY(tmp.alloc(&cl, (size_t)(kept > 0 ? kept : 1)));
  if (nnz > 0) {
    dedup_compact_k<<<grid_rows((nnz + 7) / 8), kBlock, 0, s>>>(nnz, ecol, keepf, kidx, cl);
    PRGB_LAUNCH();
  }
  *rp_out = rp;
  *col_out = cl;
  *nnz_out = kept;
  return PR_OK;
}

static unsigned grid_rows(int64_t n) {
  int64_t warps_per_block = kBlock / 32;
  int64_t g = (n + warps_per_block - 1) / warps_per_block;
  int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

pr_status ingest(const pr_csr* csr, uint32_t flags, DevGraph* g, Arena& keep, Arena& tmp, Ctl* ctl) {
  cudaStream_t s = tmp.stream();
  const int32_t n = csr->n;
  int64_t nnz = csr->nnz;
  g->n = n;
  const int32_t* rowptr = csr->rowptr;
  const int32_t* col = csr->col;
  if (csr->on_host) {
    int32_t *drp = nullptr, *dcol = nullptr;
    PRGB_TRY(tmp.alloc(&drp, (size_t)n + 1));
    PRGB_TRY(tmp.alloc(&dcol, (size_t)(nnz > 0 ? nnz : 1)));
    PRGB_COPY(cudaMemcpyAsync(drp, rowptr, ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, s));
    if (nnz > 0) PRGB_COPY(cudaMemcpyAsync(dcol, col, (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
    rowptr = drp;
    col = dcol;
  }
  if (flags & PR_CANONICALIZE) {
    int32_t *crp = nullptr, *ccol = nullptr;
    PRGB_TRY(canonicalize(rowptr, col, n, nnz, tmp, ctl, &crp, &ccol, &nnz));
    rowptr = crp;
    col = ccol;
  }
  PRGB_TRY(keep.alloc(&g->outdeg, (size_t)n + 1));
  PRGB_TRY(keep.alloc(&g->optr, (size_t)n + 1));
  PRGB_TRY(keep.alloc(&g->iptr, (size_t)n + 1));
  uint8_t* has_loop = nullptr;
  PRGB_TRY(tmp.alloc(&has_loop, (size_t)n + 1));
  if (n > 0) {
    validate_ptr_k<<<grid_rows((n + 7) / 8), kBlock, 0, s>>>(rowptr, n, nnz, has_loop, ctl);
    PRGB_LAUNCH();
    validate_cols_k<<<grid_rows((nnz + kWarpEntries - 1) / kWarpEntries), kBlock, 0, s>>>(rowptr, col, n, nnz,
                                                                                          has_loop, ctl);
    PRGB_LAUNCH();
    outdeg_k<<<grid_rows((n + 7) / 8), kBlock, 0, s>>>(rowptr, n, has_loop, g->outdeg);
    PRGB_LAUNCH();
  }
  PRGB_TRY(scan_i32(g->outdeg, g->optr, n, tmp));
  // the loop-free edge count and the validation result are needed on the host
  int32_t m32 = 0;
  int err = 0;
  PRGB_CUDA(cudaMemcpyAsync(&m32, g->optr + n, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&err, &ctl->err, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  if (err) return (pr_status)err;
  g->m = m32;
  const int64_t m = g->m;
  PRGB_TRY(keep.alloc(&g->oidx, (size_t)(m > 0 ? m : 1)));
  PRGB_TRY(keep.alloc(&g->iidx, (size_t)(m > 0 ? m : 1)));
  uint32_t *kd = nullptr, *vs = nullptr, *kt = nullptr, *vt = nullptr;
  PRGB_TRY(tmp.alloc(&kd, (size_t)(m > 0 ? m : 1)));
  PRGB_TRY(tmp.alloc(&vs, (size_t)(m > 0 ? m : 1)));
  PRGB_TRY(tmp.alloc(&kt, (size_t)(m > 0 ? m : 1)));
  PRGB_TRY(tmp.alloc(&vt, (size_t)(m > 0 ? m : 1)));
  if (n > 0) {
    strip_loops_k<<<grid_rows((nnz + kWarpEntries - 1) / kWarpEntries), kBlock, 0, s>>>(rowptr, col, n, nnz, has_loop,
                                                                                        g->optr, g->oidx, kd, vs);
    PRGB_LAUNCH();
  }
  // CSR order is (source asc, target asc); a stable sort by target gives
  // each column's sources in ascending order, and the sorted targets the
  // column offsets.
  PRGB_TRY(radix_sort_pairs(kd, vs, kt, vt, m, bits_for((uint32_t)(n > 0 ? n - 1 : 0)), tmp));
  if (m > 0) PRGB_CUDA(cudaMemcpyAsync(g->iidx, vs, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
  col_ptr_k<<<grid_rows((m + 1 + 7) / 8), kBlock, 0, s>>>(m, kd, n, g->iptr);
  PRGB_LAUNCH();
  PRGB_TRY(build_heavy(g->iptr, n, keep, tmp, &g->heavy_rows, &g->heavy_choff, &g->heavy_chrow, &g->nheavy,
                        &g->nchunks));
  PRGB_TRY(build_lorder(g->iptr, n, nullptr, 0, keep, tmp, &g->lorder));
  PRGB_TRY(build_lpre(g->iptr, g->lorder, n, g->m, keep, tmp, &g->lpre));
  // vertices with many out-edges: the partitioner spreads their chunks over warps
  PRGB_TRY(build_heavy(g->optr, n, keep, tmp, &g->oheavy, &g->ochoff, &g->ochrow, &g->noheavy, &g->nochunks));
  PRGB_TRY(build_inv(g->outdeg, n, keep, &g->inv, s));
  return PR_OK;
}

}  // namespace prgb
