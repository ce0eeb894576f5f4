// C ABI entry points: handle lifecycle, mesh setup (minimum-rule DOF numbering and element
// classes), supports, numbering queries, and dispatch to the kernel translation units.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "mto_internal.cuh"

using namespace mto;

mto_status mto_fail(mto_handle h, mto_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

mto_status mto_cuda_check(mto_handle h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MTO_OK;
  cudaGetLastError();   // do not leave a recoverable error behind for the next launch check
  return mto_fail(h, MTO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

StreamJoin::StreamJoin(mto_handle h_) : h(h_) {
  cudaSetDevice(h->device);
  cudaEventRecord(h->ev_in, h->user_stream);
  cudaStreamWaitEvent(h->stream, h->ev_in, 0);
}

StreamJoin::~StreamJoin() {
  cudaEventRecord(h->ev_out, h->stream);
  cudaStreamWaitEvent(h->user_stream, h->ev_out, 0);
}

mto_status mto_after_launch(mto_handle h, const char* what) {
  h->launches++;
  return mto_cuda_check(h, cudaGetLastError(), what);
}

namespace {
cudaEvent_t take_event(mto_handle h) {
  if (!h->timing.pool.empty()) {
    cudaEvent_t e = h->timing.pool.back();
    h->timing.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

TimedScope::TimedScope(mto_handle h_, int fam_) : h(h_), fam(fam_), launches0(h_->launches) {
  if (!h->timing.on) return;
  if (h->timing.sampled && !h->timing.sample && !(fam == F_APPLYLEAD && h->timing.sample_lead)) return;
  if (!h->timing.capture_list && h->timing.pending.size() > 4096) {
    cudaStreamSynchronize(h->stream);
    timing_harvest(h);
  }
  a = take_event(h);
  if (h->timing.capture_list) cudaEventRecordWithFlags(a, h->stream, cudaEventRecordExternal);
  else cudaEventRecord(a, h->stream);
}

TimedScope::~TimedScope() {
  if (!a) return;
  cudaEvent_t b = take_event(h);
  if (h->timing.capture_list) cudaEventRecordWithFlags(b, h->stream, cudaEventRecordExternal);
  else cudaEventRecord(b, h->stream);
  Timing::Pending pd{fam, (int)(h->launches - launches0), a, b};
  if (h->timing.capture_list) h->timing.capture_list->push_back(pd);
  else h->timing.pending.push_back(pd);
}

void graph_timing_harvest(mto_handle h, GraphEntry* g) {
  for (auto& p : g->events) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      h->timing.ms[p.fam] += ms;
      h->timing.launches[p.fam] += p.launches;
    } else {
      cudaGetLastError();
    }
  }
}

GraphEntry* find_graph(mto_handle h, const GraphKey& k) {
  for (auto* g : h->graphs)
    if (g->key == k) return g;
  return nullptr;
}

GraphEntry* new_graph(mto_handle h, const GraphKey& k) {
  if (h->graphs.size() >= 8) {
    GraphEntry* old = h->graphs.front();
    if (old->exec) cudaGraphExecDestroy(old->exec);
    for (auto& p : old->events) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    delete old;
    h->graphs.erase(h->graphs.begin());
  }
  GraphEntry* g = new GraphEntry();
  g->key = k;
  h->graphs.push_back(g);
  return g;
}

void clear_graphs(mto_handle h) {
  for (auto* g : h->graphs) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    for (auto& p : g->events) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    delete g;
  }
  h->graphs.clear();
}

void timing_harvest(mto_handle h) {
  for (auto& p : h->timing.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      h->timing.ms[p.fam] += ms;
      h->timing.launches[p.fam] += p.launches;
    } else {
      cudaGetLastError();
    }
    h->timing.pool.push_back(p.a);
    h->timing.pool.push_back(p.b);
  }
  h->timing.pending.clear();
}

namespace {

template <typename T>
void free_dev(mto_handle h, T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void release_mesh(mto_handle h) {
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  clear_graphs(h);
  free_dev(h, h->p_d);
  free_dev(h, h->d_d);
  free_dev(h, h->design_off_d);
  free_dev(h, h->cons_d);
  for (auto& c : h->pc) {
    free_dev(h, c.elem);
    free_dev(h, c.gmap);
    free_dev(h, c.dpos);
    free_dev(h, c.posc);
    free_dev(h, c.K64);
    free_dev(h, c.K32);
    free_dev(h, c.K32lo);
    free_dev(h, c.B64);
    free_dev(h, c.B32);
    free_dev(h, c.B32lo);
    c = PClass();
  }
  for (auto* v : {&h->bc, &h->bc_qr}) {
    for (auto& b : *v) {
      free_dev(h, b.elem);
      free_dev(h, b.slot);
      free_dev(h, b.K0T);
      free_dev(h, b.stab);
      free_dev(h, b.stabf);
      free_dev(h, b.tcB);
      free_dev(h, b.tcTau);
    }
    v->clear();
  }
  for (auto& q : h->qr) {
    free_dev(h, q.R);
    q = QRTab();
  }
  free_dev(h, h->slot_d);
  mg_release(h);
  for (double** v : {&h->diag64, &h->invd64, &h->r64, &h->p64, &h->s64, &h->u64, &h->w64, &h->cg_part})
    free_dev(h, *v);
  for (float** v : {&h->invd32, &h->x32, &h->r32, &h->p32, &h->s32, &h->u32, &h->w32}) free_dev(h, *v);
  h->schwarz_valid = false;
  free_dev(h, h->ibuf);
  free_dev(h, h->dbuf);
  free_dev(h, h->edge_buf);
  if (h->basis_tab) cudaFree(h->basis_tab);
  h->basis_tab = nullptr;
  h->have_setup = h->have_supports = false;
  h->built_precision = -1;
  h->k0_nu = -2.0;
  h->fixed_host.clear();
  free_dev(h, h->fixed_d);
  h->n_fixed = 0;
  free_dev(h, h->spring_dof_d);
  free_dev(h, h->spring_k_d);
  h->n_springs = 0;
  free_dev(h, h->filt_W);
  free_dev(h, h->oc_t);
  h->bytes = h->base_bytes;
}

// ---- numbering (host, integer) ---------------------------------------------------------------
inline int64_t vertex_id(mto_handle h, int ix, int iy) { return (int64_t)iy * (h->nelx + 1) + ix; }

// Global nodes of a horizontal (dir = 0) or vertical (dir = 1) edge in parameter order
// (left->right / bottom->top): start vertex, interior nodes, end vertex.  Returns the edge order.
int edge_nodes(mto_handle h, int dir, int ix, int iy, int64_t* out) {
  int pE;
  int64_t base;
  int64_t v0, v1;
  if (dir == 0) {
    int64_t id = (int64_t)iy * h->nelx + ix;
    pE = h->pH[id];
    base = h->h_base[id];
    v0 = vertex_id(h, ix, iy);
    v1 = vertex_id(h, ix + 1, iy);
  } else {
    int64_t id = (int64_t)iy * (h->nelx + 1) + ix;
    pE = h->pV[id];
    base = h->v_base[id];
    v0 = vertex_id(h, ix, iy);
    v1 = vertex_id(h, ix, iy + 1);
  }
  out[0] = v0;
  for (int k = 1; k < pE; ++k) out[k] = base + (k - 1);
  out[pE] = v1;
  return pE;
}

// (node, weight) list of local node (a, b) of element e; returns the count.
int local_node_map(mto_handle h, int64_t e, int a, int b, int64_t* nodes, double* w) {
  int ex = (int)(e % h->nelx), ey = (int)(e / h->nelx);
  int p = h->p_host[e];
  bool xa = (a == 0 || a == p), yb = (b == 0 || b == p);
  if (xa && yb) {
    nodes[0] = vertex_id(h, ex + a / p, ey + b / p);
    w[0] = 1.0;
    return 1;
  }
  if (yb || xa) {
    int64_t en[kPMaxTab + 2];
    int pE, t;
    if (yb) {
      pE = edge_nodes(h, 0, ex, ey + b / p, en);
      t = a;
    } else {
      pE = edge_nodes(h, 1, ex + a / p, ey, en);
      t = b;
    }
    if (pE == p) {
      nodes[0] = en[t];
      w[0] = 1.0;
      return 1;
    }
    double zp[kPMaxTab + 1], ze[kPMaxTab + 1];
    gll_nodes(p, zp);
    gll_nodes(pE, ze);
    for (int k = 0; k <= pE; ++k) {
      nodes[k] = en[k];
      w[k] = lagrange_val(ze, pE + 1, k, zp[t]);
    }
    return pE + 1;
  }
  nodes[0] = h->i_base[e] + (int64_t)(b - 1) * (p - 1) + (a - 1);
  w[0] = 1.0;
  return 1;
}

}  // namespace

namespace {
// f[dof[k]] += val[k] (distinct DOFs)
__global__ void scatter_add_kernel(int n, const int64_t* __restrict__ dof, const double* __restrict__ val,
                                   double* __restrict__ f) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) f[dof[k]] += val[k];
}

// Gauss-Lobatto-Legendre weights of order p: w_k = 2 / (p (p + 1) P_p(z_k)^2)
void gll_weights(int p, double* w) {
  double z[kPMaxTab + 1];
  gll_nodes(p, z);
  for (int k = 0; k <= p; ++k) {
    double pn, pn1;
    legendre_pair(p, z[k], &pn, &pn1);
    w[k] = 2.0 / (p * (p + 1) * pn * pn);
  }
}
}  // namespace

int mto::local_node_map_public(mto_handle h, int64_t e, int a, int b, int64_t* nodes, double* w) {
  return local_node_map(h, e, a, b, nodes, w);
}

extern "C" {

mto_status mto_create(mto_handle* out, int device, void* stream) {
  if (!out) return MTO_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MTO_ECUDA;
  mto_handle h = new mto_handle_s();
  h->device = device;
  h->user_stream = (cudaStream_t)stream;
  // MTO_NO_GRAPHS=1 launches the PCG iterations one kernel at a time instead of replaying captured
  // graphs (same kernels and arithmetic; for profilers that handle graphs poorly)
  if (const char* ng = std::getenv("MTO_NO_GRAPHS")) h->use_graphs = !(ng[0] == '1');
  // MTO_SOLVE_LOG=1 prints, per refinement step of mto_solve, the inner iterations, the FP64
  // relative residual and the host wall time to stderr (diagnostics; no effect on the arithmetic)
  if (const char* sl = std::getenv("MTO_SOLVE_LOG")) h->solve_log = sl[0] == '1';
  // multigrid smoothing knobs for studies of the cycle (defaults: interval ratio 100, Q1 degree 4)
  if (const char* mr = std::getenv("MTO_MG_RATIO")) h->mg_ratio = std::atof(mr);
  if (const char* md = std::getenv("MTO_MG_Q1DEG")) h->mg_q1deg = std::min(std::max(std::atoi(md), 0), 16);
  // MTO_OP_KERNEL=0 / 1 / 2 selects the split operator's kernel for n_e <= 32 as
  // mto_set_operator_kernel does (register pipeline / bulk-copy staging / generic)
  if (const char* ok = std::getenv("MTO_OP_KERNEL"))
    h->op_kernel = (ok[0] >= '0' && ok[0] <= '2') ? ok[0] - '0' : -1;
  cudaSetDevice(device);
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    delete h;
    return MTO_ECUDA;
  }
  if (mto_alloc(h, &h->red, 64) || mto_alloc(h, &h->eng, 128) || mto_alloc(h, &h->flags, 64) || mto_alloc(h, &h->sel, 256) ||
      mto_alloc(h, &h->cg_res, 64) || mto_alloc(h, &h->cg_cnt, 64) || mto_alloc(h, &h->cg_base, 4)) {
    delete h;
    return MTO_ENOMEM;
  }
  h->base_bytes = h->bytes;
  if (cudaMallocHost((void**)&h->host_pinned, 64 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&h->host_flags, 16 * sizeof(int)) != cudaSuccess) {
    delete h;
    return MTO_ENOMEM;
  }
  *out = h;
  return MTO_OK;
}

mto_status mto_destroy(mto_handle h) {
  if (!h) return MTO_OK;
  release_mesh(h);
  timing_harvest(h);
  for (cudaEvent_t e : h->timing.pool) cudaEventDestroy(e);
  cudaFree(h->cg_res);
  cudaFree(h->cg_cnt);
  cudaFree(h->cg_base);
  cudaFreeHost(h->host_flags);
  cudaStreamSynchronize(h->stream);
  cudaStreamDestroy(h->stream);
  cudaEventDestroy(h->ev_in);
  cudaEventDestroy(h->ev_out);
  cudaFree(h->red);
  cudaFree(h->eng);
  cudaFree(h->flags);
  cudaFree(h->sel);
  cudaFreeHost(h->host_pinned);
  delete h;
  return MTO_OK;
}

const char* mto_last_error(mto_handle h) { return h ? h->err.c_str() : "null handle"; }

mto_status mto_set_stream(mto_handle h, void* stream) {
  if (!h) return MTO_EINVAL;
  h->user_stream = (cudaStream_t)stream;
  return MTO_OK;
}

mto_status mto_setup(mto_handle h, int32_t nelx, int32_t nely, double hx, double hy,
                     const int32_t* p_map, const int32_t* d_map, int64_t* ndof, int64_t* design_len) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h) return MTO_EINVAL;
  h->err.clear();
  if (nelx < 1 || nely < 1 || !(hx > 0) || !(hy > 0) || !p_map || !d_map)
    return mto_fail(h, MTO_EINVAL, "mto_setup: bad mesh arguments");
  int64_t nel = (int64_t)nelx * nely;
  for (int64_t e = 0; e < nel; ++e) {
    if (p_map[e] < 1 || p_map[e] > MTO_P_MAX)
      return mto_fail(h, MTO_EINVAL, "mto_setup: p outside 1..MTO_P_MAX at element " + std::to_string(e));
    if (d_map[e] < 1 || d_map[e] > MTO_D_MAX)
      return mto_fail(h, MTO_EINVAL, "mto_setup: d outside 1..MTO_D_MAX at element " + std::to_string(e));
  }
  cudaSetDevice(h->device);
  release_mesh(h);
  h->nelx = nelx;
  h->nely = nely;
  h->hx = hx;
  h->hy = hy;
  h->nel = nel;
  h->p_host.assign(p_map, p_map + nel);
  h->d_host.assign(d_map, d_map + nel);

  // edge orders (minimum rule) and node bases
  h->pH.assign((size_t)(nely + 1) * nelx, 0);
  h->pV.assign((size_t)nely * (nelx + 1), 0);
  for (int iy = 0; iy <= nely; ++iy)
    for (int ix = 0; ix < nelx; ++ix) {
      int below = iy > 0 ? p_map[(int64_t)(iy - 1) * nelx + ix] : 1 << 20;
      int above = iy < nely ? p_map[(int64_t)iy * nelx + ix] : 1 << 20;
      h->pH[(int64_t)iy * nelx + ix] = std::min(below, above);
    }
  for (int iy = 0; iy < nely; ++iy)
    for (int ix = 0; ix <= nelx; ++ix) {
      int left = ix > 0 ? p_map[(int64_t)iy * nelx + ix - 1] : 1 << 20;
      int right = ix < nelx ? p_map[(int64_t)iy * nelx + ix] : 1 << 20;
      h->pV[(int64_t)iy * (nelx + 1) + ix] = std::min(left, right);
    }
  int64_t next = (int64_t)(nelx + 1) * (nely + 1);
  h->h_base.resize(h->pH.size());
  for (size_t k = 0; k < h->pH.size(); ++k) {
    h->h_base[k] = next;
    next += h->pH[k] - 1;
  }
  h->v_base.resize(h->pV.size());
  for (size_t k = 0; k < h->pV.size(); ++k) {
    h->v_base[k] = next;
    next += h->pV[k] - 1;
  }
  h->i_base.resize(nel);
  for (int64_t e = 0; e < nel; ++e) {
    h->i_base[e] = next;
    next += (int64_t)(p_map[e] - 1) * (p_map[e] - 1);
  }
  h->n_nodes = next;
  h->ndof = 2 * next;
  if (h->ndof >= (int64_t)1 << 31) return mto_fail(h, MTO_EINVAL, "mto_setup: more than 2^31 DOFs");
  h->design_off_host.resize(nel + 1);
  h->design_off_host[0] = 0;
  for (int64_t e = 0; e < nel; ++e)
    h->design_off_host[e + 1] = h->design_off_host[e] + (int64_t)d_map[e] * d_map[e];
  h->design_len = h->design_off_host[nel];

  // element classes by order: node maps with minimum-rule constraint records
  std::vector<Constraint> cons;
  std::vector<int> slot_of(nel, -1);
  for (int p = 1; p <= MTO_P_MAX; ++p) {
    std::vector<int> elems;
    for (int64_t e = 0; e < nel; ++e)
      if (p_map[e] == p) elems.push_back((int)e);
    PClass& c = h->pc[p];
    c.p = p;
    c.n = (int)elems.size();
    if (c.n == 0) continue;
    c.ld = round_up(c.n, 32);
    int ne = 2 * (p + 1) * (p + 1);
    c.P = packed_size(ne);
    c.L = diag_row_len(ne);
    int nn = (p + 1) * (p + 1);
    std::vector<int> gmap((size_t)nn * c.ld, 0);
    // positions of each packed entry (i <= j) in the circulant-diagonal row
    std::vector<int2> dpos(c.P);
    for (int ii = 0, cc = 0; ii < ne; ++ii)
      for (int jj = ii; jj < ne; ++jj, ++cc) {
        const int k = jj - ii;
        if (2 * k < ne) dpos[cc] = make_int2(k * ne + ii, -1);
        else if (2 * k == ne) dpos[cc] = make_int2(k * ne + ii, k * ne + jj);
        else dpos[cc] = make_int2((ne - k) * ne + jj, -1);
      }
    for (int k = 0; k < c.n; ++k) {
      int64_t e = elems[k];
      slot_of[e] = k;
      for (int b = 0; b <= p; ++b)
        for (int a = 0; a <= p; ++a) {
          int64_t nodes[kConsMax];
          double w[kConsMax];
          int cnt = local_node_map(h, e, a, b, nodes, w);
          int ln = b * (p + 1) + a;
          if (cnt == 1) {
            gmap[(size_t)k * nn + ln] = (int)nodes[0];
          } else {
            Constraint r;
            memset(&r, 0, sizeof(r));
            r.cnt = cnt;
            for (int j = 0; j < cnt; ++j) {
              r.node[j] = (int)nodes[j];
              r.w[j] = w[j];
            }
            gmap[(size_t)k * nn + ln] = -(1 + (int)cons.size());
            cons.push_back(r);
          }
        }
    }
    MTO_TRY(mto_alloc(h, &c.elem, c.n));
    MTO_TRY(mto_alloc(h, &c.gmap, gmap.size()));
    std::vector<int> posc(c.L, 0);
    for (int cc = 0; cc < c.P; ++cc) {
      posc[dpos[cc].x] = cc;
      if (dpos[cc].y >= 0) posc[dpos[cc].y] = cc;
    }
    MTO_TRY(mto_alloc(h, &c.posc, posc.size()));
    MTO_TRY(mto_cuda_check(h, cudaMemcpy(c.posc, posc.data(), posc.size() * sizeof(int), cudaMemcpyHostToDevice), "upload"));
    MTO_TRY(mto_alloc(h, &c.dpos, dpos.size()));
    MTO_TRY(mto_cuda_check(h, cudaMemcpy(c.dpos, dpos.data(), dpos.size() * sizeof(int2), cudaMemcpyHostToDevice), "upload"));
    MTO_TRY(mto_cuda_check(h, cudaMemcpy(c.elem, elems.data(), c.n * sizeof(int), cudaMemcpyHostToDevice), "upload"));
    MTO_TRY(mto_cuda_check(h, cudaMemcpy(c.gmap, gmap.data(), gmap.size() * sizeof(int), cudaMemcpyHostToDevice), "upload"));
  }
  h->n_cons = (int)cons.size();
  if (h->n_cons) {
    MTO_TRY(mto_alloc(h, &h->cons_d, cons.size()));
    MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->cons_d, cons.data(), cons.size() * sizeof(Constraint), cudaMemcpyHostToDevice), "upload"));
  }

  // (p, d) classes for the build / sensitivity, and (p+1, d) tables for the QR indicator
  for (int p = 1; p <= MTO_P_MAX; ++p)
    for (int d = 1; d <= MTO_D_MAX; ++d) {
      std::vector<int> elems, slots;
      for (int64_t e = 0; e < nel; ++e)
        if (p_map[e] == p && d_map[e] == d) {
          elems.push_back((int)e);
          slots.push_back(slot_of[e]);
        }
      if (elems.empty()) continue;
      BClass b;
      b.p = p;
      b.d = d;
      b.S = d * d;
      b.P = packed_size(2 * (p + 1) * (p + 1));
      b.n = (int)elems.size();
      MTO_TRY(mto_alloc(h, &b.elem, b.n));
      MTO_TRY(mto_alloc(h, &b.slot, b.n));
      MTO_TRY(mto_cuda_check(h, cudaMemcpy(b.elem, elems.data(), b.n * sizeof(int), cudaMemcpyHostToDevice), "upload"));
      MTO_TRY(mto_cuda_check(h, cudaMemcpy(b.slot, slots.data(), b.n * sizeof(int), cudaMemcpyHostToDevice), "upload"));
      h->bc.push_back(b);
      BClass q = b;
      q.p = p + 1;
      q.P = packed_size(2 * (p + 2) * (p + 2));
      q.elem = nullptr;
      q.slot = nullptr;
      h->bc_qr.push_back(q);
    }

  // per-element arrays
  MTO_TRY(mto_alloc(h, &h->p_d, nel));
  MTO_TRY(mto_alloc(h, &h->d_d, nel));
  MTO_TRY(mto_alloc(h, &h->design_off_d, nel + 1));
  MTO_TRY(mto_alloc(h, &h->slot_d, nel));   // slot of each element within its order class
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->p_d, p_map, nel * sizeof(int), cudaMemcpyHostToDevice), "upload"));
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->d_d, d_map, nel * sizeof(int), cudaMemcpyHostToDevice), "upload"));
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->design_off_d, h->design_off_host.data(), (nel + 1) * sizeof(int64_t), cudaMemcpyHostToDevice), "upload"));
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->slot_d, slot_of.data(), nel * sizeof(int), cudaMemcpyHostToDevice), "upload"));

  // solver workspace
  int64_t n = h->ndof;
  for (double** v : {&h->diag64, &h->invd64, &h->r64, &h->p64, &h->s64, &h->u64, &h->w64}) MTO_TRY(mto_alloc(h, v, n));
  for (float** v : {&h->invd32, &h->x32, &h->r32, &h->p32, &h->s32, &h->u32, &h->w32}) MTO_TRY(mto_alloc(h, v, n));
  // CG block partials: per launch the largest grid of a vector kernel (4 partials per block in the
  // residual kernel) or of one class's operator launch
  int64_t maxgrid = 152 * 4 * 4;
  for (int p = 1; p <= MTO_P_MAX; ++p)
    if (h->pc[p].n && ebe_blocks(p, h->pc[p].n) > maxgrid) maxgrid = ebe_blocks(p, h->pc[p].n);
  h->cg_class_stride = maxgrid;
  h->cg_stride = 8 * maxgrid;
  MTO_TRY(mto_alloc(h, &h->cg_part, (size_t)8 * h->cg_stride));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->cg_cnt, 0, 64 * sizeof(unsigned), h->stream), "memset"));
  MTO_TRY(mto_alloc(h, &h->ibuf, 4 * nel + 64));
  MTO_TRY(mto_alloc(h, &h->dbuf, 2 * nel + 64));
  h->n_edges = (int64_t)(nely + 1) * nelx + (int64_t)nely * (nelx + 1);
  MTO_TRY(mto_alloc(h, &h->edge_buf, h->n_edges + nel));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->flags, 0, 64 * sizeof(int), h->stream), "memset"));
  MTO_TRY(build_tables(h));
  MTO_TRY(build_sens_tables(h));
  MTO_TRY(mg_setup(h));
  MTO_TRY(mg_set_masks(h));
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "mto_setup"));
  h->have_setup = true;
  if (ndof) *ndof = h->ndof;
  if (design_len) *design_len = h->design_len;
  return MTO_OK;
}

mto_status mto_set_supports(mto_handle h, const int64_t* fixed, int64_t n) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h || !h->have_setup) return mto_fail(h, MTO_EINVAL, "mto_set_supports: call mto_setup first");
  if (n < 0 || (n > 0 && !fixed)) return mto_fail(h, MTO_EINVAL, "mto_set_supports: bad arguments");
  for (int64_t k = 0; k < n; ++k)
    if (fixed[k] < 0 || fixed[k] >= h->ndof)
      return mto_fail(h, MTO_EINVAL, "mto_set_supports: DOF index out of range");
  h->fixed_host.assign(fixed, fixed + n);
  std::sort(h->fixed_host.begin(), h->fixed_host.end());
  h->fixed_host.erase(std::unique(h->fixed_host.begin(), h->fixed_host.end()), h->fixed_host.end());
  free_dev(h, h->fixed_d);
  h->n_fixed = (int64_t)h->fixed_host.size();
  if (h->n_fixed) {
    MTO_TRY(mto_alloc(h, &h->fixed_d, h->n_fixed));
    MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->fixed_d, h->fixed_host.data(), h->n_fixed * sizeof(int64_t),
                                         cudaMemcpyHostToDevice), "upload"));
  }
  h->have_supports = true;
  h->schwarz_valid = false;
  MTO_TRY(mg_set_masks(h));
  if (h->built_precision >= 0) MTO_TRY(build_diagonal(h, h->built_precision));
  return MTO_OK;
}

mto_status mto_set_springs(mto_handle h, const int64_t* dofs, const double* k, int64_t n) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup) return mto_fail(h, MTO_EINVAL, "mto_set_springs: call mto_setup first");
  if (n < 0 || n > 1024 || (n > 0 && (!dofs || !k))) return mto_fail(h, MTO_EINVAL, "mto_set_springs: bad arguments");
  std::vector<std::pair<int64_t, double>> sp;
  for (int64_t i = 0; i < n; ++i) {
    if (dofs[i] < 0 || dofs[i] >= h->ndof || !(k[i] > 0) || !std::isfinite(k[i]))
      return mto_fail(h, MTO_EINVAL, "mto_set_springs: DOF out of range or stiffness not positive");
    sp.push_back({dofs[i], k[i]});
  }
  // one entry per DOF (stiffnesses on the same DOF add up)
  std::sort(sp.begin(), sp.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  std::vector<int64_t> d;
  std::vector<double> kk;
  for (const auto& e : sp) {
    if (!d.empty() && d.back() == e.first) kk.back() += e.second;
    else {
      d.push_back(e.first);
      kk.push_back(e.second);
    }
  }
  cudaSetDevice(h->device);
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "mto_set_springs"));
  clear_graphs(h);   // captured iterations hold the previous operator
  free_dev(h, h->spring_dof_d);
  free_dev(h, h->spring_k_d);
  h->n_springs = (int)d.size();
  if (h->n_springs) {
    MTO_TRY(mto_alloc(h, &h->spring_dof_d, d.size()));
    MTO_TRY(mto_alloc(h, &h->spring_k_d, kk.size()));
    MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->spring_dof_d, d.data(), d.size() * sizeof(int64_t), cudaMemcpyHostToDevice), "upload"));
    MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->spring_k_d, kk.data(), kk.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));
  }
  h->schwarz_valid = false;
  h->mg_valid = false;
  if (h->built_precision >= 0 && h->have_supports) MTO_TRY(build_diagonal(h, h->built_precision));
  return MTO_OK;
}

mto_status mto_vertex_dof(mto_handle h, int32_t ix, int32_t iy, int32_t comp, int64_t* dof) {
  if (!h || !h->have_setup || !dof) return mto_fail(h, MTO_EINVAL, "mto_vertex_dof: bad arguments");
  if (ix < 0 || ix > h->nelx || iy < 0 || iy > h->nely || comp < 0 || comp > 1)
    return mto_fail(h, MTO_EINVAL, "mto_vertex_dof: vertex or component out of range");
  *dof = 2 * vertex_id(h, ix, iy) + comp;
  return MTO_OK;
}

mto_status mto_side_dofs_in(mto_handle h, int32_t side, int32_t comp, double s0, double s1, int64_t* out,
                            int64_t cap, int64_t* count) {
  if (!h || !h->have_setup || !count) return mto_fail(h, MTO_EINVAL, "mto_side_dofs: bad arguments");
  if (side < 0 || side > 3 || comp < -1 || comp > 1) return mto_fail(h, MTO_EINVAL, "mto_side_dofs: bad side/comp");
  // nodes of the side in order with their coordinate along it (GLL positions of each edge's order)
  std::vector<int64_t> nodes;
  std::vector<double> pos;
  int64_t en[kPMaxTab + 2];
  double z[kPMaxTab + 1];
  const bool vert = side <= 1;
  const int nE = vert ? h->nely : h->nelx;
  const double len = vert ? h->hy : h->hx;
  for (int t = 0; t < nE; ++t) {
    const int pE = vert ? edge_nodes(h, 1, side == 0 ? 0 : h->nelx, t, en) : edge_nodes(h, 0, t, side == 2 ? 0 : h->nely, en);
    gll_nodes(pE, z);
    for (int k = 0; k < pE; ++k) {
      nodes.push_back(en[k]);
      pos.push_back((t + 0.5 * (1.0 + z[k])) * len);
    }
  }
  nodes.push_back(vert ? vertex_id(h, side == 0 ? 0 : h->nelx, h->nely) : vertex_id(h, h->nelx, side == 2 ? 0 : h->nely));
  pos.push_back(nE * len);
  std::vector<int64_t> dofs;
  for (size_t i = 0; i < nodes.size(); ++i) {
    if (!(pos[i] >= s0 && pos[i] <= s1)) continue;
    if (comp != 1) dofs.push_back(2 * nodes[i]);
    if (comp != 0) dofs.push_back(2 * nodes[i] + 1);
  }
  std::sort(dofs.begin(), dofs.end());
  dofs.erase(std::unique(dofs.begin(), dofs.end()), dofs.end());
  *count = (int64_t)dofs.size();
  if (cap > 0) {
    if (!out) return mto_fail(h, MTO_EINVAL, "mto_side_dofs: null output");
    int64_t m = std::min<int64_t>(cap, (int64_t)dofs.size());
    std::copy(dofs.begin(), dofs.begin() + m, out);
  }
  return MTO_OK;
}

mto_status mto_side_dofs(mto_handle h, int32_t side, int32_t comp, int64_t* out, int64_t cap, int64_t* count) {
  return mto_side_dofs_in(h, side, comp, -HUGE_VAL, HUGE_VAL, out, cap, count);
}

mto_status mto_edge_dofs(mto_handle h, int32_t dir, int32_t ix, int32_t iy, int32_t comp, int64_t* out, int64_t cap,
                         int64_t* count) {
  if (!h || !h->have_setup || !count || comp < 0 || comp > 1 || (dir != 0 && dir != 1))
    return mto_fail(h, MTO_EINVAL, "mto_edge_dofs: bad arguments");
  if (dir == 0 ? (ix < 0 || ix >= h->nelx || iy < 0 || iy > h->nely) : (ix < 0 || ix > h->nelx || iy < 0 || iy >= h->nely))
    return mto_fail(h, MTO_EINVAL, "mto_edge_dofs: edge out of range");
  int64_t en[kPMaxTab + 2];
  const int pE = edge_nodes(h, dir, ix, iy, en);
  *count = pE + 1;
  if (cap > 0) {
    if (!out) return mto_fail(h, MTO_EINVAL, "mto_edge_dofs: null output");
    for (int k = 0; k <= pE && k < cap; ++k) out[k] = 2 * en[k] + comp;
  }
  return MTO_OK;
}

mto_status mto_side_load(mto_handle h, int32_t side, int32_t comp, double traction, double* f) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup || !f || side < 0 || side > 3 || comp < 0 || comp > 1 || !std::isfinite(traction))
    return mto_fail(h, MTO_EINVAL, "mto_side_load: bad arguments");
  cudaSetDevice(h->device);
  // accumulate per node on the host (vertices are shared by two edges), then one scatter
  std::vector<std::pair<int64_t, double>> acc;
  const bool vert = side <= 1;
  const int nE = vert ? h->nely : h->nelx;
  const double len = vert ? h->hy : h->hx;
  for (int t = 0; t < nE; ++t) {
    int64_t en[kPMaxTab + 2];
    const int pE = vert ? edge_nodes(h, 1, side == 0 ? 0 : h->nelx, t, en) : edge_nodes(h, 0, t, side == 2 ? 0 : h->nely, en);
    double w[kPMaxTab + 1];
    gll_weights(pE, w);
    for (int k = 0; k <= pE; ++k) acc.push_back({2 * en[k] + comp, traction * 0.5 * len * w[k]});
  }
  std::sort(acc.begin(), acc.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  std::vector<int64_t> dofs;
  std::vector<double> vals;
  for (const auto& kv : acc) {
    if (!dofs.empty() && dofs.back() == kv.first) vals.back() += kv.second;
    else {
      dofs.push_back(kv.first);
      vals.push_back(kv.second);
    }
  }
  const int n = (int)dofs.size();
  int64_t* d_dof = nullptr;
  double* d_val = nullptr;
  MTO_TRY(mto_cuda_check(h, cudaMalloc(&d_dof, n * sizeof(int64_t)), "cudaMalloc"));
  mto_status st = mto_cuda_check(h, cudaMalloc(&d_val, n * sizeof(double)), "cudaMalloc");
  if (st == MTO_OK)
    st = mto_cuda_check(h, cudaMemcpyAsync(d_dof, dofs.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream), "copy");
  if (st == MTO_OK)
    st = mto_cuda_check(h, cudaMemcpyAsync(d_val, vals.data(), n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy");
  if (st == MTO_OK) {
    scatter_add_kernel<<<(n + 255) / 256, 256, 0, h->stream>>>(n, d_dof, d_val, f);
    st = mto_after_launch(h, "scatter_add_kernel");
  }
  if (st == MTO_OK) st = mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  cudaFree(d_dof);
  cudaFree(d_val);
  return st;
}

mto_status mto_element_nodes(mto_handle h, int64_t e, int64_t* nodes, double* weights, int32_t* counts) {
  if (!h || !h->have_setup || !nodes || !weights || !counts || e < 0 || e >= h->nel)
    return mto_fail(h, MTO_EINVAL, "mto_element_nodes: bad arguments");
  int p = h->p_host[e];
  for (int b = 0; b <= p; ++b)
    for (int a = 0; a <= p; ++a) {
      int ln = b * (p + 1) + a;
      counts[ln] = local_node_map(h, e, a, b, nodes + ln * kConsMax, weights + ln * kConsMax);
    }
  return MTO_OK;
}

mto_status mto_build_elements(mto_handle h, const double* rho, const mto_material* mat, int32_t precision) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h || !h->have_setup || !rho || !mat) return mto_fail(h, MTO_EINVAL, "mto_build_elements: bad arguments");
  if (precision != MTO_FP64 && precision != MTO_MIXED) return mto_fail(h, MTO_EINVAL, "mto_build_elements: bad precision");
  if (!(mat->E0 > 0) || !(mat->Emin >= 0) || !(mat->nu > -1 && mat->nu < 0.5) || !(mat->q >= 1))
    return mto_fail(h, MTO_EINVAL, "mto_build_elements: bad material");
  cudaSetDevice(h->device);
  h->built_precision = precision;
  h->schwarz_valid = false;
  h->mg_valid = false;
  MTO_TRY(build_elements(h, rho, mat, precision));
  if (h->have_supports) MTO_TRY(build_diagonal(h, precision));
  return MTO_OK;
}

mto_status mto_element_matrix(mto_handle h, int64_t e, double* packed) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h || !h->have_setup || !packed || e < 0 || e >= h->nel)
    return mto_fail(h, MTO_EINVAL, "mto_element_matrix: bad arguments");
  if (h->built_precision < 0) return mto_fail(h, MTO_EINVAL, "mto_element_matrix: call mto_build_elements first");
  cudaSetDevice(h->device);
  return element_matrix(h, e, packed);
}

mto_status mto_solve(mto_handle h, const double* f, double* u, const mto_solve_opts* opts, int32_t* iters,
                     double* relres) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h || !h->have_setup || !f || !u || !opts) return mto_fail(h, MTO_EINVAL, "mto_solve: bad arguments");
  if (!h->have_supports) return mto_fail(h, MTO_EINVAL, "mto_solve: call mto_set_supports first");
  if (h->built_precision < 0) return mto_fail(h, MTO_EINVAL, "mto_solve: call mto_build_elements first");
  if (opts->precision != MTO_FP64 && opts->precision != MTO_MIXED && opts->precision != MTO_MIXED32)
    return mto_fail(h, MTO_EINVAL, "mto_solve: bad precision");
  if (opts->norm != MTO_NORM_L2 && opts->norm != MTO_NORM_JACOBI && opts->norm != MTO_NORM_ENERGY)
    return mto_fail(h, MTO_EINVAL, "mto_solve: bad norm");
  if (opts->norm == MTO_NORM_ENERGY && opts->precision == MTO_MIXED32)
    return mto_fail(h, MTO_EINVAL, "mto_solve: the compliance-accuracy test needs FP64 vectors");
  if (opts->precision != MTO_FP64 && h->built_precision != MTO_MIXED)
    return mto_fail(h, MTO_EINVAL, "mto_solve: the mixed solves need the split-precision (MTO_MIXED) build");
  if (!(opts->rtol > 0) || opts->max_iter < 1 || opts->check_every < 1 ||
      (opts->precond != MTO_PREC_JACOBI && opts->precond != MTO_PREC_SCHWARZ && opts->precond != MTO_PREC_MG))
    return mto_fail(h, MTO_EINVAL, "mto_solve: bad options");
  cudaSetDevice(h->device);
  return solve(h, f, u, opts, iters, relres);
}

namespace {
// common checks of one instance of a batched call
mto_status batch_check(mto_handle h, int device, const char* what) {
  if (!h) return MTO_EINVAL;
  if (h->device != device) return mto_fail(h, MTO_EINVAL, std::string(what) + ": handles on different devices");
  if (!h->have_setup) return mto_fail(h, MTO_EINVAL, std::string(what) + ": call mto_setup first");
  return MTO_OK;
}
}  // namespace

mto_status mto_build_elements_batched(mto_handle* hs, int32_t n, const double* const* rho, const mto_material* mat,
                                      int32_t precision) {
  if (!hs || n < 1 || !rho || !mat) return MTO_EINVAL;
  mto_status first = MTO_OK;
  for (int32_t i = 0; i < n; ++i) {   // asynchronous on every handle's own stream
    const mto_status st = mto_build_elements(hs[i], rho[i], mat, precision);
    if (first == MTO_OK && st != MTO_OK) first = st;
  }
  return first;
}

mto_status mto_solve_batched(mto_handle* hs, int32_t n, const double* const* f, double* const* u,
                             const mto_solve_opts* opts, int32_t* iters, double* relres, mto_status* status) {
  if (!hs || n < 1 || !f || !u || !opts || !hs[0]) return MTO_EINVAL;
  const int device = hs[0]->device;
  for (int32_t i = 0; i < n; ++i) {
    MTO_TRY(batch_check(hs[i], device, "mto_solve_batched"));
    mto_handle h = hs[i];
    if (!f[i] || !u[i]) return mto_fail(h, MTO_EINVAL, "mto_solve_batched: bad arguments");
    if (!h->have_supports) return mto_fail(h, MTO_EINVAL, "mto_solve_batched: call mto_set_supports first");
    if (h->built_precision < 0) return mto_fail(h, MTO_EINVAL, "mto_solve_batched: call mto_build_elements first");
    if (opts->precision != MTO_FP64 && opts->precision != MTO_MIXED)
      return mto_fail(h, MTO_EINVAL, "mto_solve_batched: precision MTO_FP64 or MTO_MIXED");
    if (opts->precision == MTO_MIXED && h->built_precision != MTO_MIXED)
      return mto_fail(h, MTO_EINVAL, "mto_solve_batched: the mixed solve needs the MTO_MIXED build");
    for (int32_t k = 0; k < i; ++k)
      if (hs[k] == h) return mto_fail(h, MTO_EINVAL, "mto_solve_batched: a handle appears twice");
  }
  if (!(opts->rtol > 0) || opts->max_iter < 1 || opts->check_every < 1 ||
      (opts->precond != MTO_PREC_JACOBI && opts->precond != MTO_PREC_SCHWARZ && opts->precond != MTO_PREC_MG) ||
      (opts->norm != MTO_NORM_L2 && opts->norm != MTO_NORM_JACOBI && opts->norm != MTO_NORM_ENERGY))
    return mto_fail(hs[0], MTO_EINVAL, "mto_solve_batched: bad options");
  cudaSetDevice(device);
  std::vector<std::unique_ptr<StreamJoin>> joins;
  for (int32_t i = 0; i < n; ++i) joins.emplace_back(new StreamJoin(hs[i]));
  return solve_batched(hs, n, f, u, opts, iters, relres, status);
}

mto_status mto_sensitivity_batched(mto_handle* hs, int32_t n, const double* const* u, const double* const* f,
                                   const double* const* rho, const mto_material* mat, double* const* dc, double* C) {
  if (!hs || n < 1 || !u || !f || !rho || !mat || !dc) return MTO_EINVAL;
  mto_status first = MTO_OK;
  for (int32_t i = 0; i < n; ++i) {   // the launches of every instance first (asynchronous) ...
    const mto_status st = mto_sensitivity(hs[i], u[i], f[i], rho[i], mat, MTO_FP64, dc[i], nullptr);
    if (first == MTO_OK && st != MTO_OK) first = st;
  }
  if (first != MTO_OK || !C) return first;
  for (int32_t i = 0; i < n; ++i) {   // ... then the compliances (one synchronisation each)
    mto_handle h = hs[i];
    MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->host_pinned + 8, h->red + 8, sizeof(double), cudaMemcpyDeviceToHost,
                                              h->stream), "copy"));
  }
  for (int32_t i = 0; i < n; ++i) {
    mto_handle h = hs[i];
    MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
    C[i] = h->host_pinned[8];
  }
  return MTO_OK;
}

mto_status mto_apply(mto_handle h, const double* x, double* y) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h || !h->have_setup || !x || !y) return mto_fail(h, MTO_EINVAL, "mto_apply: bad arguments");
  if (h->built_precision < 0) return mto_fail(h, MTO_EINVAL, "mto_apply: call mto_build_elements first");
  cudaSetDevice(h->device);
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(y, 0, h->ndof * sizeof(double), h->stream), "mto_apply"));
  return apply64(h, x, y);
}

mto_status mto_compliance(mto_handle h, const double* f, const double* u, double* C_dev, double* C) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup || !f || !u || (!C_dev && !C)) return mto_fail(h, MTO_EINVAL, "mto_compliance: bad arguments");
  cudaSetDevice(h->device);
  double* out = C_dev ? C_dev : h->red + 9;
  MTO_TRY(dot64(h, f, u, h->ndof, out));
  if (!C) return MTO_OK;
  MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->host_pinned + 40, out, sizeof(double), cudaMemcpyDeviceToHost,
                                            h->stream), "copy"));
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  *C = h->host_pinned[40];
  return MTO_OK;
}

mto_status mto_compliance_energy(mto_handle h, const double* u, const double* f, const double* rho,
                                 const mto_material* mat, double* C) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup || !u || !f || !rho || !mat || !C)
    return mto_fail(h, MTO_EINVAL, "mto_compliance_energy: bad arguments");
  cudaSetDevice(h->device);
  return compliance_energy(h, u, f, rho, mat, C);
}

mto_status mto_apply_operator(mto_handle h, int32_t op, const double* x, double* y, double* xKx) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup || !x || !y) return mto_fail(h, MTO_EINVAL, "mto_apply_operator: bad arguments");
  if (op != MTO_OP_FP64 && op != MTO_OP_SPLIT && op != MTO_OP_LEAD)
    return mto_fail(h, MTO_EINVAL, "mto_apply_operator: bad operator");
  if (h->built_precision < 0) return mto_fail(h, MTO_EINVAL, "mto_apply_operator: call mto_build_elements first");
  if (op != MTO_OP_FP64 && h->built_precision != MTO_MIXED)
    return mto_fail(h, MTO_EINVAL, "mto_apply_operator: the split operator needs the MTO_MIXED build");
  cudaSetDevice(h->device);
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(y, 0, h->ndof * sizeof(double), h->stream), "mto_apply_operator"));
  return apply_operator(h, op, x, y, xKx);
}

mto_status mto_set_operator_kernel(mto_handle h, int32_t kernel) {
  if (!h) return MTO_EINVAL;
  if (kernel < MTO_OPK_AUTO || kernel > MTO_OPK_GENERIC)
    return mto_fail(h, MTO_EINVAL, "mto_set_operator_kernel: bad kernel");
  if (kernel != h->op_kernel) {
    cudaSetDevice(h->device);
    MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "mto_set_operator_kernel"));
    clear_graphs(h);   // captured iterations hold the previous kernel
  }
  h->op_kernel = kernel;
  for (auto& k : h->op_kernel_cls) k = -2;   // the explicit choice overrides the autotuner's
  return MTO_OK;
}

mto_status mto_autotune(mto_handle h, int32_t* choice, double* us) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup || h->built_precision < 0) return mto_fail(h, MTO_EINVAL, "mto_autotune: build first");
  cudaSetDevice(h->device);
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "mto_autotune"));
  return autotune_operator(h, choice, us);
}

mto_status mto_element_matrix_split(mto_handle h, int64_t e, float* hi, float* lo) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup || !hi || !lo || e < 0 || e >= h->nel)
    return mto_fail(h, MTO_EINVAL, "mto_element_matrix_split: bad arguments");
  if (h->built_precision != MTO_MIXED)
    return mto_fail(h, MTO_EINVAL, "mto_element_matrix_split: call mto_build_elements with MTO_MIXED first");
  cudaSetDevice(h->device);
  return element_matrix_split(h, e, hi, lo);
}

mto_status mto_sensitivity(mto_handle h, const double* u, const double* f, const double* rho,
                           const mto_material* mat, int32_t precision, double* dc, double* C) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h || !h->have_setup || !u || !f || !rho || !mat || !dc)
    return mto_fail(h, MTO_EINVAL, "mto_sensitivity: bad arguments");
  if (precision != MTO_FP64 && precision != MTO_MIXED) return mto_fail(h, MTO_EINVAL, "mto_sensitivity: bad precision");
  cudaSetDevice(h->device);
  return sensitivity(h, u, f, rho, mat, precision, dc, C);
}

mto_status mto_transfer_design(mto_handle h, const int32_t* d_old, const double* rho_old, double* rho_new) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup || !d_old || !rho_old || !rho_new || rho_old == rho_new)
    return mto_fail(h, MTO_EINVAL, "mto_transfer_design: bad arguments");
  cudaSetDevice(h->device);
  return transfer_design(h, d_old, rho_old, rho_new);
}

mto_status mto_filter(mto_handle h, double radius, const double* rho, double* rho_f) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup || !rho || !rho_f || rho == rho_f || !(radius > 0) || !std::isfinite(radius))
    return mto_fail(h, MTO_EINVAL, "mto_filter: bad arguments");
  if (radius > 4.0 * std::min(h->hx, h->hy)) return mto_fail(h, MTO_EINVAL, "mto_filter: radius above 4 elements");
  cudaSetDevice(h->device);
  return density_filter(h, radius, rho, rho_f, false);
}

mto_status mto_filter_adjoint(mto_handle h, double radius, const double* g_f, double* g) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup || !g_f || !g || g == g_f || !(radius > 0) || !std::isfinite(radius))
    return mto_fail(h, MTO_EINVAL, "mto_filter_adjoint: bad arguments");
  if (radius > 4.0 * std::min(h->hx, h->hy)) return mto_fail(h, MTO_EINVAL, "mto_filter_adjoint: radius above 4 elements");
  cudaSetDevice(h->device);
  return density_filter(h, radius, g_f, g, true);
}

mto_status mto_sensitivity_adjoint(mto_handle h, const double* u, const double* v, const double* rho,
                                   const mto_material* mat, double* dc) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h->have_setup || !u || !v || !rho || !mat || !dc)
    return mto_fail(h, MTO_EINVAL, "mto_sensitivity_adjoint: bad arguments");
  cudaSetDevice(h->device);
  return sensitivity_adjoint(h, u, v, rho, mat, dc);
}

mto_status mto_indicator(mto_handle h, const double* u, const double* rho, const mto_material* mat,
                         const mto_indicator_opts* opts, double* gamma_a, double* gamma_d, double* eps_qr,
                         int32_t* p_new, int32_t* d_new, int8_t* theta) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h || !h->have_setup || !u || !rho || !mat || !opts)
    return mto_fail(h, MTO_EINVAL, "mto_indicator: bad arguments");
  if (h->built_precision < 0) return mto_fail(h, MTO_EINVAL, "mto_indicator: call mto_build_elements first");
  if (opts->cycle < 1 || opts->p_max < 1 || opts->p_max > MTO_P_MAX || opts->d_max < 1 ||
      opts->d_max > MTO_D_MAX * MTO_D_MAX)
    return mto_fail(h, MTO_EINVAL, "mto_indicator: bad options");
  cudaSetDevice(h->device);
  return indicators(h, u, rho, mat, opts, gamma_a, gamma_d, eps_qr, p_new, d_new, theta);
}

mto_status mto_map_update(mto_handle h, const double* gamma_a, const double* gamma_d, const double* eps_qr,
                          const mto_indicator_opts* opts, int32_t* p_new, int32_t* d_new, int8_t* theta) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h || !h->have_setup || !gamma_a || !gamma_d || !eps_qr || !opts || !p_new || !d_new || !theta)
    return mto_fail(h, MTO_EINVAL, "mto_map_update: bad arguments");
  if (opts->p_max < 1 || opts->p_max > MTO_P_MAX || opts->d_max < 1 || opts->d_max > MTO_D_MAX * MTO_D_MAX)
    return mto_fail(h, MTO_EINVAL, "mto_map_update: bad options");
  cudaSetDevice(h->device);
  return map_update(h, gamma_a, gamma_d, eps_qr, opts, p_new, d_new, theta);
}

mto_status mto_oc_update(mto_handle h, const double* rho, const double* dc, double volfrac, double move,
                         double eta, double* rho_new, double* lambda) {
  if (!h) return MTO_EINVAL;
  StreamJoin join(h);
  if (!h || !h->have_setup || !rho || !dc || !rho_new) return mto_fail(h, MTO_EINVAL, "mto_oc_update: bad arguments");
  if (!(volfrac > 0 && volfrac <= 1) || !(move > 0) || !(eta > 0))
    return mto_fail(h, MTO_EINVAL, "mto_oc_update: bad parameters");
  cudaSetDevice(h->device);
  return oc_update(h, rho, dc, volfrac, move, eta, rho_new, lambda);
}

mto_status mto_timing_enable(mto_handle h, int32_t enable) {
  if (!h) return MTO_EINVAL;
  cudaSetDevice(h->device);
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "mto_timing_enable"));
  timing_harvest(h);
  for (int f = 0; f < F_COUNT; ++f) {
    h->timing.ms[f] = 0.0;
    h->timing.launches[f] = 0;
  }
  h->timing.on = enable != 0;
  h->timing.sampled = enable == 2;
  return MTO_OK;
}

mto_status mto_timing_read(mto_handle h, int32_t family, int64_t* launches, double* total_ms) {
  if (!h || family < 0 || family >= F_COUNT || !launches || !total_ms)
    return mto_fail(h, MTO_EINVAL, "mto_timing_read: bad arguments");
  cudaSetDevice(h->device);
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "mto_timing_read"));
  timing_harvest(h);
  *launches = h->timing.launches[family];
  *total_ms = h->timing.ms[family];
  return MTO_OK;
}

mto_status mto_set_build_path(mto_handle h, int32_t path) {
  if (!h || (path != MTO_BUILD_TENSOR && path != MTO_BUILD_SIMT))
    return mto_fail(h, MTO_EINVAL, "mto_set_build_path: bad path");
  h->build_path = path;
  return MTO_OK;
}

mto_status mto_memory(mto_handle h, int64_t* bytes) {
  if (!h || !bytes) return MTO_EINVAL;
  *bytes = h->bytes;
  return MTO_OK;
}

mto_status mto_launch_count(mto_handle h, int64_t* count) {
  if (!h || !count) return MTO_EINVAL;
  *count = h->launches;
  return MTO_OK;
}

}  // extern "C"
