// Products over many HODLRdD trees in one launch per stage (a "forest"): the
// batched use of the hierarchical product (many independent kernel matrices
// of uneven size, one product K v each per iteration, as in the paper's
// kernel-SVM experiment), for handles of the tensor-core form (FP16X2).
//
// At creation the trees' packed factor planes are copied into one stream (one
// tensor map), their V and U panels into one panel list each (row, column, t
// and output indices shifted by each tree's offsets), their near-field tasks
// into one task list per pass (with per-task coordinate and point bases, scale
// and diagonal), and the persistent CTAs' panel ranges are balanced over the
// whole forest. A product is then one gather, one V-apply, one U-apply (and the
// sum of cut panels), one near-field launch per pass and one final sum, for
// all trees together; the results equal the trees' own products (the same
// arithmetic on the same data, up to the summation of the near field's chunk
// sums, which follows the same order).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"

namespace hd {
namespace {

struct TreeInfo {
  int64_t off;   // first point of the tree in the forest's tree-ordered rows
  int64_t xoff;  // first element of its N x nrhs input / output
  int64_t yoff;  // first row of its level slices
  int32_t N, nrhs, kappa, pad;
};
static_assert(sizeof(TreeInfo) == 40, "TreeInfo layout");

// x_t[p][c] = x_tree[perm[p] * nrhs + c] for c < nrhs (0 beyond), and the
// column maxima of |x_t| over the forest.
__global__ void k_forest_gather(int64_t Ntot, const int32_t* __restrict__ tp, const TreeInfo* __restrict__ ti,
                                const int32_t* __restrict__ perm, const float* __restrict__ xin,
                                float* __restrict__ xt, unsigned int* __restrict__ colmax) {
  __shared__ unsigned int smax[kTcR];
  if (threadIdx.x < kTcR) smax[threadIdx.x] = 0u;
  __syncthreads();
  const int c = threadIdx.x % kTcR;
  unsigned int m = 0u;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < Ntot * kTcR;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / kTcR;
    const TreeInfo T = ti[tp[p]];
    const float v = c < T.nrhs ? xin[T.xoff + (int64_t)perm[p] * T.nrhs + c] : 0.f;
    xt[e] = v;
    m = max(m, __float_as_uint(fabsf(v)));
  }
  atomicMax(&smax[c], m);
  __syncthreads();
  if (threadIdx.x < kTcR) atomicMax(&colmax[threadIdx.x], smax[threadIdx.x]);
}

// y_tree[perm[p] * nrhs + c] = near(p, c) + the tree's level slices at p.
__global__ void k_forest_finish(int64_t Ntot, const int32_t* __restrict__ tp, const TreeInfo* __restrict__ ti,
                                const int32_t* __restrict__ perm, const float* __restrict__ ynear,
                                const float* __restrict__ ylev, float* __restrict__ yout) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < Ntot * kTcR;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / kTcR;
    const int c = (int)(e % kTcR);
    const TreeInfo T = ti[tp[p]];
    if (c >= T.nrhs) continue;
    const int64_t local = p - T.off;
    float acc = ynear[e];
    for (int l = 0; l < T.kappa; ++l) acc += ylev[(T.yoff + (int64_t)l * T.N + local) * kTcR + c];
    yout[T.xoff + (int64_t)perm[p] * T.nrhs + c] = acc;
  }
}

}  // namespace
}  // namespace hd

struct hodlrdd_forest_s {
  int device = 0;
  int d = 0, kid = 0;
  float kc = 0.f;
  std::vector<hodlrdd_s*> h;
  std::vector<int> nrhs;
  std::vector<hd::TreeInfo> info;
  int64_t Ntot = 0, xtot = 0, ylev_rows = 0, trank = 0;
  hd::DevBuf<int32_t> tp, perm;
  hd::DevBuf<hd::TreeInfo> dinfo;
  hd::DevBuf<float> xin, yout, xt, t, ylev, ynear, pbuf;
  hd::DevBuf<int32_t> err;
  hd::TcStream v, u;
  hd::DevBuf<int32_t> vmap, splitp;
  hd::DevBuf<float> fac, wbox;
  hd::DevBuf<int2> split;
  int64_t nsplit = 0, parts = 0;
  // near field: tasks of all trees, one range per pass
  hd::DevBuf<int4> ntasks, nsrcs;
  hd::DevBuf<float4> nsoff, nhi, nlo;
  hd::DevBuf<int2> nbase;
  hd::DevBuf<float2> nsd;
  hd::DevBuf<int2> ntbox;      // per task: its box records (packed small boxes)
  hd::DevBuf<int32_t> nbrow;
  hd::DevBuf<float4> nboff;
  hd::DevBuf<uint32_t> nemask;  // per source entry
  std::vector<std::pair<int64_t, int64_t>> passes;
  cudaStream_t st = nullptr, aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int64_t launches = 0;
  // the schedules' fixed cost per panel, picked by timing at creation
  double fixed_v = 32768.0, fixed_u = 32768.0;
  cudaGraphExec_t graph = nullptr;  // one run's launches, captured once
};

namespace hd {
namespace {

void forest_free(hodlrdd_forest_s* f) {
  if (!f) return;
  if (f->st) cudaStreamSynchronize(f->st);
  if (f->aux) cudaStreamSynchronize(f->aux);
  if (f->ev_fork) cudaEventDestroy(f->ev_fork);
  if (f->ev_join) cudaEventDestroy(f->ev_join);
  if (f->graph) cudaGraphExecDestroy(f->graph);
  cudaStream_t st = f->st, aux = f->aux;
  delete f;
  if (st) cudaStreamDestroy(st);
  if (aux) cudaStreamDestroy(aux);
}

template <class T>
int download_all(std::vector<T>& out, const DevBuf<T>& d, cudaStream_t st) {
  out.resize(d.n);
  if (d.n) HD_CUDA(cudaMemcpyAsync(out.data(), d.p, d.n * sizeof(T), cudaMemcpyDeviceToHost, st));
  return HODLRDD_OK;
}

// The forest's panels, planes and tables from its trees' tensor-core data.
int forest_build(hodlrdd_forest_s* f) {
  cudaStream_t st = f->st;
  const int n = (int)f->h.size();
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device);
  // offsets
  std::vector<int64_t> toff(n), vcol(n), wb(n), part(n), rowv(n), rowu(n), panu(n);
  int64_t a_pts = 0, a_x = 0, a_y = 0, a_t = 0, a_vc = 0, a_wb = 0, a_part = 0, a_rv = 0, a_ru = 0, a_pu = 0;
  f->info.resize(n);
  for (int i = 0; i < n; ++i) {
    const hodlrdd_s* h = f->h[i];
    const Plan& P = h->plan;
    TreeInfo& T = f->info[i];
    T.off = a_pts;
    T.xoff = a_x;
    T.yoff = a_y;
    T.N = (int32_t)h->N;
    T.nrhs = f->nrhs[i];
    T.kappa = h->kappa;
    T.pad = 0;
    toff[i] = a_t;
    vcol[i] = a_vc;
    wb[i] = a_wb;
    part[i] = a_part;
    rowv[i] = a_rv;
    rowu[i] = a_ru;
    panu[i] = a_pu;
    a_pts += h->N;
    a_x += h->N * f->nrhs[i];
    a_y += (int64_t)h->kappa * h->N;
    a_t += h->total_rank;
    a_vc += (int64_t)P.tc_vmap.n;
    a_wb += (int64_t)P.tc_wbox.n;
    a_part += P.tc_parts;
    a_rv += P.tcv.rows;
    a_ru += P.tcu.rows;
    a_pu += (int64_t)P.tcu.h_panels.size();
  }
  f->Ntot = a_pts;
  f->xtot = a_x;
  f->ylev_rows = a_y;
  f->trank = a_t;
  f->parts = a_part;
  if (a_pts >= INT32_MAX || a_t >= INT32_MAX || a_y >= INT32_MAX || a_vc >= INT32_MAX || a_rv >= INT32_MAX - 64 ||
      a_ru >= INT32_MAX - 64) {
    set_error("hodlrdd_forest_create: the trees together exceed the 32-bit indices of the tensor-core form");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  // per point: its tree and its local original index
  {
    std::vector<int32_t> tp((size_t)a_pts), perm((size_t)a_pts);
    for (int i = 0; i < n; ++i)
      for (int64_t p = 0; p < f->h[i]->N; ++p) {
        tp[f->info[i].off + p] = i;
        perm[f->info[i].off + p] = f->h[i]->h_perm[p];
      }
    HD_TRY(upload(f->tp, tp, st));
    HD_TRY(upload(f->perm, perm, st));
    HD_TRY(upload(f->dinfo, f->info, st));
  }
  // factor planes: the trees' streams one after another
  HD_TRY(f->v.data.alloc((size_t)std::max<int64_t>(a_rv, 1) * 64));
  HD_TRY(f->u.data.alloc((size_t)std::max<int64_t>(a_ru, 1) * 64));
  f->v.rows = a_rv;
  f->u.rows = a_ru;
  HD_TRY(f->fac.alloc(std::max<int64_t>(a_t, 1)));
  HD_TRY(f->wbox.alloc(std::max<int64_t>(a_wb, 1)));
  std::vector<int32_t> vmap;
  vmap.reserve((size_t)a_vc);
  for (int i = 0; i < n; ++i) {
    const hodlrdd_s* h = f->h[i];
    const Plan& P = h->plan;
    if (P.tcv.rows)
      HD_CUDA(cudaMemcpyAsync(f->v.data.p + rowv[i] * 64, P.tcv.data.p, (size_t)P.tcv.rows * 128,
                              cudaMemcpyDeviceToDevice, st));
    if (P.tcu.rows)
      HD_CUDA(cudaMemcpyAsync(f->u.data.p + rowu[i] * 64, P.tcu.data.p, (size_t)P.tcu.rows * 128,
                              cudaMemcpyDeviceToDevice, st));
    if (h->total_rank)
      HD_CUDA(cudaMemcpyAsync(f->fac.p + toff[i], P.tc_fac.p, (size_t)h->total_rank * sizeof(float),
                              cudaMemcpyDeviceToDevice, st));
    if (P.tc_wbox.n)
      HD_CUDA(cudaMemcpyAsync(f->wbox.p + wb[i], P.tc_wbox.p, P.tc_wbox.n * sizeof(float), cudaMemcpyDeviceToDevice,
                              st));
    std::vector<int32_t> vm;
    HD_TRY(download_all(vm, P.tc_vmap, st));
    HD_CUDA(cudaStreamSynchronize(st));
    for (int32_t c : vm) vmap.push_back(c + (int32_t)toff[i]);
    // V panels: x_t rows, V columns and stream rows shift by the tree's offsets
    for (TcPanel Q : P.tcv.h_panels) {
      Q.arow += rowv[i];
      Q.brow += (int32_t)f->info[i].off;
      Q.out0 += (int32_t)vcol[i];
      f->v.h_panels.push_back(Q);
    }
    // U panels: t rows and stream rows shift; the output row names the tree's slice directly
    for (TcPanel Q : P.tcu.h_panels) {
      Q.arow += rowu[i];
      Q.brow += (int32_t)toff[i];
      Q.out0 = (int32_t)(f->info[i].yoff + (int64_t)Q.slice * h->N + Q.out0);
      Q.slice = 0;
      Q.sbox += (int32_t)wb[i];
      if (Q.part >= 0) Q.part += (int32_t)part[i];
      f->u.h_panels.push_back(Q);
    }
  }
  std::vector<int2> split;
  std::vector<int32_t> splitp;
  for (int i = 0; i < n; ++i) {
    const Plan& P = f->h[i]->plan;
    for (size_t k = 0; k < P.h_tc_split.size(); ++k) {
      split.push_back(make_int2(P.h_tc_split[k].x + (int32_t)part[i], P.h_tc_split[k].y));
      splitp.push_back(P.h_tc_splitp[k] + (int32_t)panu[i]);
    }
  }
  f->nsplit = (int64_t)split.size();
  tc_schedule_stream(f->v, sms);
  tc_schedule_stream(f->u, sms);
  HD_TRY(upload(f->v.panels, f->v.h_panels.empty() ? std::vector<TcPanel>{TcPanel{}} : f->v.h_panels, st));
  HD_TRY(upload(f->u.panels, f->u.h_panels.empty() ? std::vector<TcPanel>{TcPanel{}} : f->u.h_panels, st));
  HD_TRY(upload(f->v.cta, f->v.h_cta, st));
  HD_TRY(upload(f->u.cta, f->u.h_cta, st));
  HD_TRY(upload(f->vmap, vmap.empty() ? std::vector<int32_t>{0} : vmap, st));
  HD_TRY(upload(f->split, split.empty() ? std::vector<int2>{make_int2(0, 0)} : split, st));
  HD_TRY(upload(f->splitp, splitp.empty() ? std::vector<int32_t>{0} : splitp, st));
  HD_TRY(tc_encode_tmap(f->v));
  HD_TRY(tc_encode_tmap(f->u));
  return HODLRDD_OK;
}

// Near-field tasks of all trees: pass k holds the k-th task range of every tree
// (its coarse dense levels, the subtracted leaf blocks, the leaf pass), so that
// no two tasks of one launch write the same row; within a pass the tasks are
// sorted by work. Every (tree, level) coordinate array the tasks read is
// copied once into the forest's coordinate arrays.
int forest_near(hodlrdd_forest_s* f) {
  cudaStream_t st = f->st;
  const int n = (int)f->h.size();
  struct Range {
    int level;
    int64_t t0, t1;
    float scale, diag;
  };
  std::vector<std::vector<Range>> ranges(n);
  size_t npass = 0;
  for (int i = 0; i < n; ++i) {
    const hodlrdd_s* h = f->h[i];
    const Plan& P = h->plan;
    const float ks = (float)h->K.scale, kd = (float)h->K.diag;
    for (const DenseLevel& DL : P.coarse4) ranges[i].push_back({DL.level, DL.t0, DL.t1, ks, 0.f});
    if (P.excl4.t1 > P.excl4.t0) ranges[i].push_back({P.excl4.level, P.excl4.t0, P.excl4.t1, -ks, 0.f});
    ranges[i].push_back({P.leaf4.level, P.leaf4.t0, P.leaf4.t1, ks, kd});
    npass = std::max(npass, ranges[i].size());
  }
  // coordinates: one copy per (tree, level)
  std::vector<std::vector<int64_t>> cbase(n);
  int64_t ncoord = 0;
  for (int i = 0; i < n; ++i) {
    cbase[i].assign(f->h[i]->kappa + 1, -1);
    for (const Range& R : ranges[i])
      if (cbase[i][R.level] < 0) {
        cbase[i][R.level] = ncoord;
        ncoord += f->h[i]->N;
      }
  }
  HD_TRY(f->nhi.alloc(std::max<int64_t>(ncoord, 1)));
  HD_TRY(f->nlo.alloc(std::max<int64_t>(ncoord, 1)));
  for (int i = 0; i < n; ++i)
    for (int l = 0; l <= f->h[i]->kappa; ++l)
      if (cbase[i][l] >= 0) {
        const Plan& P = f->h[i]->plan;
        HD_CUDA(cudaMemcpyAsync(f->nhi.p + cbase[i][l], P.hi4[l].p, f->h[i]->N * sizeof(float4),
                                cudaMemcpyDeviceToDevice, st));
        HD_CUDA(cudaMemcpyAsync(f->nlo.p + cbase[i][l], P.lo4[l].p, f->h[i]->N * sizeof(float4),
                                cudaMemcpyDeviceToDevice, st));
      }
  // tasks and their sources
  std::vector<int4> tasks, srcs;
  std::vector<float4> soff;
  std::vector<int2> base;
  std::vector<float2> sd;
  std::vector<std::vector<int4>> t4(n), s4(n);
  std::vector<std::vector<float4>> o4(n), bo4(n);
  std::vector<std::vector<int2>> tb4(n);
  std::vector<std::vector<int32_t>> br4(n);
  std::vector<std::vector<uint32_t>> em4(n);
  std::vector<int64_t> soff_at(n), rec_at(n);
  for (int i = 0; i < n; ++i) {
    const Plan& P = f->h[i]->plan;
    HD_TRY(download_all(t4[i], P.tasks4, st));
    HD_TRY(download_all(s4[i], P.srcs4, st));
    HD_TRY(download_all(o4[i], P.soff4, st));
    HD_TRY(download_all(tb4[i], P.tbox4, st));
    HD_TRY(download_all(br4[i], P.brow4, st));
    HD_TRY(download_all(bo4[i], P.boff4, st));
    HD_TRY(download_all(em4[i], P.emask4, st));
  }
  HD_CUDA(cudaStreamSynchronize(st));
  std::vector<uint32_t> emask;
  std::vector<int32_t> brow;
  std::vector<float4> boff;
  for (int i = 0; i < n; ++i) {
    soff_at[i] = (int64_t)srcs.size();
    srcs.insert(srcs.end(), s4[i].begin(), s4[i].end());
    soff.insert(soff.end(), o4[i].begin(), o4[i].end());
    // a tree without packing tables: one box per task, every entry read by it
    if (tb4[i].size() != t4[i].size()) {
      tb4[i].clear();
      br4[i].clear();
      bo4[i].clear();
      for (size_t t = 0; t < t4[i].size(); ++t) {
        tb4[i].push_back(make_int2((int32_t)t, 1));
        br4[i].push_back(0);
        bo4[i].push_back(make_float4(0.f, 0.f, 0.f, 0.f));
      }
    }
    if (em4[i].size() != s4[i].size()) em4[i].assign(s4[i].size(), ~0u);
    emask.insert(emask.end(), em4[i].begin(), em4[i].end());
    rec_at[i] = (int64_t)brow.size();
    brow.insert(brow.end(), br4[i].begin(), br4[i].end());
    boff.insert(boff.end(), bo4[i].begin(), bo4[i].end());
  }
  if ((int64_t)srcs.size() >= INT32_MAX || (int64_t)brow.size() >= INT32_MAX) {
    set_error("hodlrdd_forest_create: too many near-field sources");
    return HODLRDD_ERR_UNSUPPORTED;
  }
  std::vector<int2> tbox;
  f->passes.clear();
  for (size_t k = 0; k < npass; ++k) {
    std::vector<std::pair<int64_t, size_t>> order;  // (-work, index into the pass's entries)
    std::vector<int4> pt;
    std::vector<int2> pb, ptb;
    std::vector<float2> ps;
    for (int i = 0; i < n; ++i) {
      if (k >= ranges[i].size()) continue;
      const Range& R = ranges[i][k];
      for (int64_t t = R.t0; t < R.t1; ++t) {
        int4 T = t4[i][t];
        int64_t work = 0;
        for (int32_t e = T.z; e < T.w; ++e) work += s4[i][e].y;
        T.z += (int32_t)soff_at[i];
        T.w += (int32_t)soff_at[i];
        order.push_back({-(int64_t)T.y * work, pt.size()});
        pt.push_back(T);
        pb.push_back(make_int2((int32_t)cbase[i][R.level], (int32_t)f->info[i].off));
        ps.push_back(make_float2(R.scale, R.diag));
        ptb.push_back(make_int2(tb4[i][t].x + (int32_t)rec_at[i], tb4[i][t].y));
      }
    }
    std::stable_sort(order.begin(), order.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    const int64_t t0 = (int64_t)tasks.size();
    for (const auto& o : order) {
      tasks.push_back(pt[o.second]);
      base.push_back(pb[o.second]);
      sd.push_back(ps[o.second]);
      tbox.push_back(ptb[o.second]);
    }
    f->passes.push_back({t0, (int64_t)tasks.size()});
  }
  HD_TRY(upload(f->ntasks, tasks.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : tasks, st));
  HD_TRY(upload(f->nsrcs, srcs.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : srcs, st));
  HD_TRY(upload(f->nsoff, soff.empty() ? std::vector<float4>{make_float4(0, 0, 0, 0)} : soff, st));
  HD_TRY(upload(f->nbase, base.empty() ? std::vector<int2>{make_int2(0, 0)} : base, st));
  HD_TRY(upload(f->nsd, sd.empty() ? std::vector<float2>{make_float2(0, 0)} : sd, st));
  HD_TRY(upload(f->ntbox, tbox.empty() ? std::vector<int2>{make_int2(0, 1)} : tbox, st));
  HD_TRY(upload(f->nbrow, brow.empty() ? std::vector<int32_t>{0} : brow, st));
  HD_TRY(upload(f->nboff, boff.empty() ? std::vector<float4>{make_float4(0, 0, 0, 0)} : boff, st));
  HD_TRY(upload(f->nemask, emask.empty() ? std::vector<uint32_t>{~0u} : emask, st));
  return HODLRDD_OK;
}

int forest_workspace(hodlrdd_forest_s* f) {
  HD_TRY(f->xin.alloc(std::max<int64_t>(f->xtot, 1)));
  HD_TRY(f->yout.alloc(std::max<int64_t>(f->xtot, 1)));
  HD_TRY(f->xt.alloc((size_t)f->Ntot * kTcR));
  HD_TRY(f->t.alloc((size_t)std::max<int64_t>(f->trank, 1) * kTcR));
  HD_TRY(f->ylev.alloc((size_t)std::max<int64_t>(f->ylev_rows, 1) * kTcR));
  HD_TRY(f->ynear.alloc((size_t)f->Ntot * kTcR));
  HD_TRY(f->pbuf.alloc(((size_t)std::max<int64_t>(f->parts, 1) * 128 + 1) * kTcR));
  HD_TRY(f->err.alloc(1));
  HD_CUDA(cudaMemsetAsync(f->err.p, 0, sizeof(int32_t), f->st));
  HD_CUDA(cudaStreamSynchronize(f->st));
  return HODLRDD_OK;
}

// One product of every tree on f->st (the near field on f->aux).
int forest_launch(hodlrdd_forest_s* f, cudaEvent_t* ev = nullptr) {
  cudaStream_t st = f->st;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device);
  unsigned int* colmax = reinterpret_cast<unsigned int*>(f->pbuf.p + (size_t)std::max<int64_t>(f->parts, 1) * 128 * kTcR);
  const int grid = (int)std::min<int64_t>((f->Ntot * kTcR + 255) / 256, (int64_t)sms * 16);
  if (ev) HD_CUDA(cudaEventRecord(ev[0], st));
  HD_CUDA(cudaMemsetAsync(colmax, 0, kTcR * sizeof(unsigned int), st));
  k_forest_gather<<<grid, 256, 0, st>>>(f->Ntot, f->tp.p, f->dinfo.p, f->perm.p, f->xin.p, f->xt.p, colmax);
  HD_CUDA(cudaGetLastError());
  if (ev) HD_CUDA(cudaEventRecord(ev[1], st));
  HD_CUDA(cudaEventRecord(f->ev_fork, st));
  HD_CUDA(cudaMemsetAsync(f->ylev.p, 0, (size_t)std::max<int64_t>(f->ylev_rows, 1) * kTcR * sizeof(float), st));
  TcLaunch lv{&f->v, f->xt.p, colmax, f->vmap.p, f->fac.p, f->wbox.p, f->t.p, nullptr, f->Ntot};
  HD_TRY(launch_tc_stage(true, lv, f->err.p, st));
  if (ev) HD_CUDA(cudaEventRecord(ev[2], st));
  HD_CUDA(cudaStreamWaitEvent(f->aux, f->ev_fork, 0));
  if (ev) HD_CUDA(cudaEventRecord(ev[4], f->aux));
  HD_CUDA(cudaMemsetAsync(f->ynear.p, 0, (size_t)f->Ntot * kTcR * sizeof(float), f->aux));
  for (const auto& ps : f->passes)
    HD_TRY(launch_tc_near_raw(f->d, f->kid, f->aux, ps.second - ps.first, f->ntasks.p + ps.first, f->nsrcs.p,
                              f->nsoff.p, f->nhi.p, f->nlo.p, f->xt.p, colmax, f->kc, f->ynear.p,
                              f->nbase.p + ps.first, f->nsd.p + ps.first,
                              TcPack{f->ntbox.p + ps.first, f->nbrow.p, f->nboff.p, f->nemask.p}, f->err.p));
  if (ev) HD_CUDA(cudaEventRecord(ev[5], f->aux));
  HD_CUDA(cudaEventRecord(f->ev_join, f->aux));
  TcLaunch lu{&f->u, f->t.p, colmax, f->vmap.p, f->fac.p, f->wbox.p, f->ylev.p, f->pbuf.p, 0};
  HD_TRY(launch_tc_stage(false, lu, f->err.p, st));
  HD_TRY(launch_tc_combine(f->nsplit, f->split.p, f->splitp.p, f->u.panels.p, f->pbuf.p, 0, f->ylev.p, st));
  if (ev) HD_CUDA(cudaEventRecord(ev[3], st));
  HD_CUDA(cudaStreamWaitEvent(st, f->ev_join, 0));
  k_forest_finish<<<grid, 256, 0, st>>>(f->Ntot, f->tp.p, f->dinfo.p, f->perm.p, f->ynear.p, f->ylev.p, f->yout.p);
  HD_CUDA(cudaGetLastError());
  if (ev) HD_CUDA(cudaEventRecord(ev[6], st));
  f->launches += 4 + (int64_t)f->passes.size() + (f->nsplit > 0 ? 1 : 0);
  return HODLRDD_OK;
}

// The autotuner: each apply stage's panel ranges are rebuilt for a few fixed
// costs per panel (the weight of a panel's hand-over against its bytes), each
// timed on the forest's own data layout (zero inputs: the arithmetic does not
// depend on the values), and the fastest kept.
int forest_tune(hodlrdd_forest_s* f) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device);
  cudaStream_t st = f->st;
  unsigned int* colmax = reinterpret_cast<unsigned int*>(f->pbuf.p + (size_t)std::max<int64_t>(f->parts, 1) * 128 * kTcR);
  HD_CUDA(cudaMemsetAsync(f->xt.p, 0, (size_t)f->Ntot * kTcR * sizeof(float), st));
  HD_CUDA(cudaMemsetAsync(f->t.p, 0, (size_t)std::max<int64_t>(f->trank, 1) * kTcR * sizeof(float), st));
  HD_CUDA(cudaMemsetAsync(colmax, 0, kTcR * sizeof(unsigned int), st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HD_CUDA(cudaEventCreate(&e0));
  HD_CUDA(cudaEventCreate(&e1));
  const double cand[4] = {8192.0, 32768.0, 131072.0, 524288.0};
  int rc = HODLRDD_OK;
  for (int stage = 0; stage < 2 && rc == HODLRDD_OK; ++stage) {
    const bool vmode = stage == 0;
    TcStream& S = vmode ? f->v : f->u;
    if (S.h_panels.empty()) continue;
    double best_ms = 1e30, best = 32768.0;
    for (double c : cand) {
      tc_schedule_stream(S, sms, c);
      rc = upload(S.cta, S.h_cta, st);
      if (rc != HODLRDD_OK) break;
      TcLaunch L = vmode ? TcLaunch{&f->v, f->xt.p, colmax, f->vmap.p, f->fac.p, f->wbox.p, f->t.p, nullptr, f->Ntot}
                         : TcLaunch{&f->u, f->t.p, colmax, f->vmap.p, f->fac.p, f->wbox.p, f->ylev.p, f->pbuf.p, 0};
      rc = launch_tc_stage(vmode, L, f->err.p, st);  // warm
      if (rc != HODLRDD_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(e0, st) != cudaSuccess) rc = HODLRDD_ERR_CUDA;
      for (int rep = 0; rep < 2 && rc == HODLRDD_OK; ++rep) rc = launch_tc_stage(vmode, L, f->err.p, st);
      if (rc == HODLRDD_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = cuda_fail(cudaGetLastError(), "forest autotuning", __FILE__, __LINE__);
      if (rc != HODLRDD_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    if (rc != HODLRDD_OK) break;
    (vmode ? f->fixed_v : f->fixed_u) = best;
    tc_schedule_stream(S, sms, best);
    rc = upload(S.cta, S.h_cta, st);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HD_TRY(rc);
  HD_CUDA(cudaStreamSynchronize(st));
  int32_t code = 0;
  HD_CUDA(cudaMemcpy(&code, f->err.p, sizeof code, cudaMemcpyDeviceToHost));
  if (code != 0) {
    cudaMemset(f->err.p, 0, sizeof code);
    set_error("hodlrdd_forest_create: a bounded device-side wait expired while tuning");
    return HODLRDD_ERR_TIMEOUT;
  }
  return HODLRDD_OK;
}

// One run's launches captured into a CUDA graph (after one eager run, which
// also sets the kernels' attributes outside the capture).
int forest_capture(hodlrdd_forest_s* f) {
  HD_TRY(forest_launch(f));
  HD_CUDA(cudaStreamSynchronize(f->st));
  cudaGraph_t g = nullptr;
  HD_CUDA(cudaStreamBeginCapture(f->st, cudaStreamCaptureModeRelaxed));
  const int rc = forest_launch(f);
  const cudaError_t e = cudaStreamEndCapture(f->st, &g);
  if (rc != HODLRDD_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "forest capture", __FILE__, __LINE__);
  const cudaError_t e2 = cudaGraphInstantiate(&f->graph, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    f->graph = nullptr;
    return cuda_fail(e2, "forest graph", __FILE__, __LINE__);
  }
  return HODLRDD_OK;
}

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" int hodlrdd_forest_create(const hodlrdd_handle* handles, const int* nrhs, int count, hodlrdd_forest* out) {
  if (!handles || !nrhs || count < 1 || !out) {
    set_error("hodlrdd_forest_create: NULL argument or count < 1");
    return HODLRDD_ERR_INVALID;
  }
  *out = nullptr;
  int dev = 0;
  HD_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < count; ++i) {
    const hodlrdd_s* h = handles[i];
    if (!h || nrhs[i] < 1 || nrhs[i] > kTcR) {
      set_error("hodlrdd_forest_create: NULL handle or nrhs outside 1..64");
      return HODLRDD_ERR_INVALID;
    }
    for (int j = 0; j < i; ++j)
      if (handles[j] == h) {
        set_error("hodlrdd_forest_create: a handle appears twice");
        return HODLRDD_ERR_INVALID;
      }
    if (h->opt.precision != HODLRDD_PREC_FP16X2 || !tc_near_supported(h) || h->device != dev) {
      set_error("hodlrdd_forest_create: every handle must be of precision FP16X2 with a bounded kernel "
                "(not 1/r, 1/r^2), d <= 4, on the current device");
      return HODLRDD_ERR_UNSUPPORTED;
    }
    if (h->d != handles[0]->d || h->K.id != handles[0]->K.id || h->K.p0 != handles[0]->K.p0 ||
        h->K.p1 != handles[0]->K.p1) {
      set_error("hodlrdd_forest_create: the trees must share d, the kernel and its shape parameters");
      return HODLRDD_ERR_UNSUPPORTED;
    }
    if (h->profiling) {
      set_error("hodlrdd_forest_create: a handle has profiling on");
      return HODLRDD_ERR_INVALID;
    }
  }
  hodlrdd_forest_s* f = new (std::nothrow) hodlrdd_forest_s();
  if (!f) return HODLRDD_ERR_OOM;
  f->device = dev;
  f->h.assign(handles, handles + count);
  f->nrhs.assign(nrhs, nrhs + count);
  f->d = handles[0]->d;
  f->kid = handles[0]->K.id;
  f->kc = (float)kernel_const(handles[0]->K);
  int rc = HODLRDD_OK;
  try {
    cudaError_t e = cudaStreamCreateWithFlags(&f->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) rc = cuda_fail(e, "forest streams", __FILE__, __LINE__);
    if (rc == HODLRDD_OK) rc = forest_build(f);
    if (rc == HODLRDD_OK) rc = forest_near(f);
    if (rc == HODLRDD_OK) rc = forest_workspace(f);
    if (rc == HODLRDD_OK) rc = forest_tune(f);
    if (rc == HODLRDD_OK) rc = forest_capture(f);
  } catch (const std::bad_alloc&) {
    set_error("hodlrdd_forest_create: host allocation failed");
    rc = HODLRDD_ERR_OOM;
  }
  if (rc != HODLRDD_OK) {
    forest_free(f);
    return rc;
  }
  *out = f;
  return HODLRDD_OK;
}

extern "C" int hodlrdd_forest_run(hodlrdd_forest f, const void* const* x, void* const* y, void* stream) {
  if (!f || !x || !y) {
    set_error("hodlrdd_forest_run: NULL argument");
    return HODLRDD_ERR_INVALID;
  }
  const int n = (int)f->h.size();
  for (int i = 0; i < n; ++i)
    if (!x[i] || !y[i]) {
      set_error("hodlrdd_forest_run: NULL x or y");
      return HODLRDD_ERR_INVALID;
    }
  int dev = 0;
  HD_CUDA(cudaGetDevice(&dev));
  if (dev != f->device) {
    set_error("hodlrdd_forest_run: the current device is not the forest's");
    return HODLRDD_ERR_INVALID;
  }
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev = nullptr;
  HD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  // the inputs after the caller's earlier work, on the forest's stream
  cudaError_t e = cudaEventRecord(ev, caller);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(f->st, ev, 0);
  for (int i = 0; i < n && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(f->xin.p + f->info[i].xoff, x[i], (size_t)f->h[i]->N * f->nrhs[i] * sizeof(float),
                        cudaMemcpyDefault, f->st);
  int rc = HODLRDD_OK;
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "hodlrdd_forest_run: inputs", __FILE__, __LINE__);
  } else {
    e = cudaGraphLaunch(f->graph, f->st);
    if (e != cudaSuccess) rc = cuda_fail(e, "hodlrdd_forest_run", __FILE__, __LINE__);
    f->launches += 4 + (int64_t)f->passes.size() + (f->nsplit > 0 ? 1 : 0);
  }
  for (int i = 0; i < n && rc == HODLRDD_OK; ++i) {
    e = cudaMemcpyAsync(y[i], f->yout.p + f->info[i].xoff, (size_t)f->h[i]->N * f->nrhs[i] * sizeof(float),
                        cudaMemcpyDefault, f->st);
    if (e != cudaSuccess) rc = cuda_fail(e, "hodlrdd_forest_run: outputs", __FILE__, __LINE__);
  }
  // synchronous: the caller's buffers may be host memory, and the bounded
  // waits' error word is read before returning
  e = cudaStreamSynchronize(f->st);
  if (rc == HODLRDD_OK && e != cudaSuccess) rc = cuda_fail(e, "hodlrdd_forest_run", __FILE__, __LINE__);
  cudaEventDestroy(ev);
  if (rc == HODLRDD_OK) {
    int32_t code = 0;
    e = cudaMemcpy(&code, f->err.p, sizeof code, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "hodlrdd_forest_run: error word", __FILE__, __LINE__);
    if (code != 0) {
      cudaMemset(f->err.p, 0, sizeof code);
      set_error("hodlrdd_forest_run: a bounded device-side wait expired; the products are invalid");
      return HODLRDD_ERR_TIMEOUT;
    }
  }
  return rc;
}

extern "C" int hodlrdd_forest_profile(hodlrdd_forest f, double* ms) {
  if (!f || !ms) {
    set_error("hodlrdd_forest_profile: NULL argument");
    return HODLRDD_ERR_INVALID;
  }
  cudaEvent_t ev[7] = {};
  int rc = HODLRDD_OK;
  for (int i = 0; i < 7 && rc == HODLRDD_OK; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "forest events", __FILE__, __LINE__);
  if (rc == HODLRDD_OK) rc = forest_launch(f, ev);
  if (rc == HODLRDD_OK) {
    const cudaError_t e = cudaStreamSynchronize(f->st);
    if (e != cudaSuccess) rc = cuda_fail(e, "hodlrdd_forest_profile", __FILE__, __LINE__);
  }
  if (rc == HODLRDD_OK) {
    const int pairs[5][2] = {{0, 1}, {1, 2}, {2, 3}, {4, 5}, {0, 6}};
    for (int k = 0; k < 5; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[pairs[k][0]], ev[pairs[k][1]]);
      ms[k] = t;
    }
  }
  for (int i = 0; i < 7; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  return rc;
}

extern "C" int hodlrdd_forest_destroy(hodlrdd_forest f) {
  forest_free(f);
  return HODLRDD_OK;
}

extern "C" int hodlrdd_forest_stats(hodlrdd_forest f, int64_t* out) {
  if (!f || !out) return HODLRDD_ERR_INVALID;
  out[0] = f->Ntot;
  out[1] = (f->v.rows + f->u.rows) * 128;  // 64 FP16 per plane row
  out[2] = (int64_t)f->v.h_panels.size() + (int64_t)f->u.h_panels.size();
  out[3] = (int64_t)f->passes.size();
  out[4] = 4 + (int64_t)f->passes.size() + (f->nsplit > 0 ? 1 : 0);
  out[5] = (int64_t)f->fixed_v;
  out[6] = (int64_t)f->fixed_u;
  return HODLRDD_OK;
}
