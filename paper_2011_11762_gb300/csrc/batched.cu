// Batched products (step S9): many independent products C_i = A_i B_i, each
// with its own plan and leaf size, in ONE persistent launch.  The work list
// concatenates every product's C leaves, ordered longest segment first across
// all products (so uneven products balance), each unit packed as
// (product << 32) | C leaf.  Creating a batch allocates every output and all
// launch tables; running it only launches, so a run can be captured in a
// CUDA graph and replayed.
#include <vector>

#include "internal.h"

namespace cht {

// Implemented in split.cu.
int split_batch_prepare(cht_batch *b, cudaStream_t s);
int split_batch_run(cht_batch *b, cudaStream_t s);
void split_batch_release(cht_batch *b);

namespace {

// Keys (longest segment first) and packed ids for one product's units.
__global__ void k_batch_units(const int64_t *__restrict__ seg, int64_t n, int64_t prod,
                              int64_t off, int lpt, uint64_t *__restrict__ key,
                              int64_t *__restrict__ packed, int32_t *__restrict__ idx) {
  for (int64_t u = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; u < n;
       u += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t len = seg[u + 1] - seg[u];
    if (len > 0xffffffffLL) len = 0xffffffffLL;
    key[off + u] = lpt ? 0xffffffffULL - static_cast<uint64_t>(len) : 0ULL;
    packed[off + u] = (prod << 32) | u;
    idx[off + u] = static_cast<int32_t>(off + u);
  }
}

__global__ void k_gather_i64(const int32_t *__restrict__ idx, const int64_t *__restrict__ in,
                             int64_t n, int64_t *__restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = in[idx[i]];
}

}  // namespace

int batch_create(int32_t count, const cht_plan_t *plans, const cht_mat_t *As, const cht_mat_t *Bs,
                 int mode, int32_t nslices, cudaStream_t s, cht_batch **out) {
  if (mode != CHT_FP64 && mode != CHT_SPLIT_BF16) {
    set_error("unknown mode %d", mode);
    return CHT_ERR_INVALID;
  }
  auto bt = std::make_unique<cht_batch>();
  bt->count = count;
  bt->mode = mode;
  bt->nslices = nslices;
  int64_t total_vals = 0, total_units = 0;
  DevArray<int> flag;
  CHT_TRY(flag.alloc(1, s));
  for (int32_t i = 0; i < count; ++i) {
    cht_plan *p = plans[i];
    cht_mat *A = As[i], *B = Bs[i];
    if (!p || !A || !B) {
      set_error("product %d: null plan or matrix", i);
      return CHT_ERR_INVALID;
    }
    if (check_plan_operands(p, A, B, flag.p, s) != CHT_OK) {
      set_error("product %d: matrices do not match the plan's operands", i);
      return CHT_ERR_SHAPE;
    }
    if (p->b != 32 && p->b != 64) {
      set_error("product %d: leaf size %d (the batched kernels take 32 or 64)", i, p->b);
      return CHT_ERR_UNSUPPORTED;
    }
    if (p->b > bt->maxb) bt->maxb = p->b;
    bt->plans.push_back(p);
    bt->As.push_back(A);
    bt->Bs.push_back(B);
    total_vals += p->C->nnz * p->b * p->b;
    total_units += p->C->nnz;
  }
  CHT_TRY(bt->cvals.alloc(total_vals, s));
  CHT_TRY(bt->counter.alloc(1, s));
  std::vector<ProdDesc> host(count);
  int64_t voff = 0;
  for (int32_t i = 0; i < count; ++i) {
    cht_plan *p = bt->plans[i];
    ProdDesc &d = host[i];
    d.X = bt->As[i]->values();
    d.Y = bt->Bs[i]->values();
    d.Z = bt->cvals.p + voff;
    d.px = p->pa.p;
    d.py = p->pb.p;
    d.seg = p->cseg.p;
    d.b = p->b;
    d.nx = bt->As[i]->pat->nnz;
    d.ny = bt->Bs[i]->pat->nnz;
    d.nz = p->C->nnz;
    d.npairs = p->npairs;
    auto v = std::make_unique<cht_mat>();
    v->pat = p->C;
    v->plan_id = p->id;
    v->view = true;
    v->view_vals = bt->cvals.p + voff;
    bt->views.push_back(std::move(v));
    voff += p->C->nnz * p->b * p->b;
  }
  CHT_TRY(bt->prods.alloc(count, s));
  CHT_CUDA_TRY(cudaMemcpyAsync(bt->prods.p, host.data(), sizeof(ProdDesc) * count,
                               cudaMemcpyHostToDevice, s));
  // the work list: every C leaf of every product, longest segment first
  bt->nunits = total_units;
  CHT_TRY(bt->units.alloc(total_units, s));
  if (total_units > 0) {
    if (total_units > 0x7fffffffLL) {
      set_error("batch has too many output leaves");
      return CHT_ERR_UNSUPPORTED;
    }
    DevArray<uint64_t> key, skey;
    DevArray<int64_t> packed;
    DevArray<int32_t> idx, sidx;
    CHT_TRY(key.alloc(total_units, s));
    CHT_TRY(skey.alloc(total_units, s));
    CHT_TRY(packed.alloc(total_units, s));
    CHT_TRY(idx.alloc(total_units, s));
    CHT_TRY(sidx.alloc(total_units, s));
    const int lpt = g_opt.schedule == 0 && mode == CHT_FP64 ? 1 : 0;
    int64_t uoff = 0;
    for (int32_t i = 0; i < count; ++i) {
      const int64_t n = bt->plans[i]->C->nnz;
      if (n > 0) {
        k_batch_units<<<grid_for(n, 256), 256, 0, s>>>(bt->plans[i]->cseg.p, n, i, uoff, lpt,
                                                       key.p, packed.p, idx.p);
        CHT_TRY(launched("batch_units"));
      }
      uoff += n;
    }
    if (lpt) CHT_TRY(radix_sort_pairs(key.p, idx.p, skey.p, sidx.p, total_units, 32, s));
    k_gather_i64<<<grid_for(total_units, 256), 256, 0, s>>>(lpt ? sidx.p : idx.p, packed.p,
                                                            total_units, bt->units.p);
    CHT_TRY(launched("gather_i64"));
  }
  if (mode == CHT_SPLIT_BF16) CHT_TRY(split_batch_prepare(bt.get(), s));
  CHT_CUDA_TRY(cudaStreamSynchronize(s));  // host tables go out of scope
  *out = bt.release();
  return CHT_OK;
}

int batch_run(cht_batch *b, cudaStream_t s) {
  if (b->mode == CHT_SPLIT_BF16) return split_batch_run(b, s);
  return launch_leafgemm_f64_batch(b->prods.p, b->count, b->units.p, b->nunits, b->maxb,
                                   b->counter.p, s);
}

int batch_output(cht_batch *b, int32_t i, cht_mat **C) {
  if (i < 0 || i >= b->count) {
    set_error("batch output %d out of range [0, %d)", i, b->count);
    return CHT_ERR_INVALID;
  }
  *C = b->views[i].get();
  return CHT_OK;
}

void batch_destroy(cht_batch *b) { delete b; }

}  // namespace cht

cht_batch::~cht_batch() { cht::split_batch_release(this); }
