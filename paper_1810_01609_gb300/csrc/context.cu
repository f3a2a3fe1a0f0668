// libmdwf host runtime: context, device workspaces, the launch autotuner, the even-odd
// operator compositions, CG on the normal equations (plain FP64 and mixed precision with
// reliable updates), CUDA-graph replay of the CG iteration, and the C ABI of mdwf.h.
//
// Solver (Sec. "Current State of the Art"): red-black preconditioned CG on the normal
// equations, "double-half": inner iterations in low-precision storage with float
// arithmetic, occasional reliable updates that recompute the residual in FP64.
#include "mdwf.h"
#include "mdwf_kernels.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <condition_variable>
#include <memory>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

using namespace mdwf;

namespace {
thread_local std::string g_last_error;

void set_err(const char* what, cudaError_t e) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  g_last_error = buf;
}
}  // namespace

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      set_err(#call, e_);                                          \
      return e_ == cudaErrorMemoryAllocation ? MDWF_ERR_OOM : MDWF_ERR_CUDA; \
    }                                                              \
  } while (0)
#define CKS(call)                                \
  do {                                           \
    int s_ = (call);                             \
    if (s_ != MDWF_SUCCESS) return s_;           \
  } while (0)

struct TuneEntry {
  int ns;
  double ms;
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct mdwf_ctx {
  mdwf_params prm;
  int device = -1;   // CUDA device current at mdwf_create: the context's buffers live there
  Geom g;
  int Ls;
  long long vh;
  double alpha5, beta5;
  // gauge: [prec][parity]
  void* gauge[NPREC][2] = {};   // [storage precision][parity]
  int gs[NPREC] = {};
  bool gauge_loaded = false;
  std::map<std::string, DevBuf> ws;
  // reductions
  double* partials = nullptr;
  size_t partials_n = 0;
  unsigned* counter = nullptr;       // grid-reduction counters: [0] and one per block group
  size_t counters_n = 0;
  double* red_out = nullptr;   // device [256]
  double* red_host = nullptr;  // pinned [256]
  CGScalars* cg = nullptr;     // device [64]
  CGScalars* cg_host = nullptr;
  int* dev_status = nullptr;   // device flag set by a kernel whose bounded wait gave up
  int* status_host = nullptr;  // pinned copy
  // tuning
  bool tuning = true;
  std::map<std::string, TuneEntry> tune;
  std::string tune_file;
  // graphs
  std::map<std::string, cudaGraphExec_t> graphs;
  std::map<std::string, double> graph_bytes;  // algorithmic bytes of one replay
  long long launches = 0;
  double bytes = 0.0;  // algorithmic HBM bytes of every kernel launched (see site_bytes)
  // T partition (t_ranks > 1): the local lattice is one slab of the global one
  long long slice_vh = 0;            // checkerboard sites of one local timeslice
  mdwf_face_exchange_fn xfn = nullptr;
  void* xuser = nullptr;
  void* user_faces[4] = {};          // caller-owned face buffers (send lo/hi, recv lo/hi)
  size_t user_face_bytes = 0;
  std::shared_ptr<void> group;       // in-process partition group this context belongs to
  // FP64 hops of the calls in progress run in emulated FP64 (double-float; set around the
  // operator applications that use it, never on a T-partitioned context)
  bool emu_active = false;
};

// emulated-FP64 hops for the lifetime of the scope (restores the previous setting)
struct EmuScope {
  mdwf_ctx* c;
  bool old;
  EmuScope(mdwf_ctx* cc, bool on) : c(cc), old(cc->emu_active) { c->emu_active = on && c->prm.t_ranks == 1; }
  ~EmuScope() { c->emu_active = old; }
};

constexpr int PREC_F64E = 5;   // MDWF_PREC_F64E: FP64 storage, emulated-FP64 hops

namespace {

// ---------------------------------------------------------------- s-operators
SOp sop_none() {
  SOp o;
  memset(&o, 0, sizeof o);
  return o;
}
// FP32 copies of the coefficients for the 32-bit kernels
static void sop_round(SOp& o) {
  o.fa = (float)o.a; o.fb = (float)o.b; o.finv_a = (float)o.inv_a; o.fc0 = (float)o.c0;
  for (int j = 0; j < MAXLS; j++) o.fw[j] = (float)o.w[j];
}
SOp sop_bidiag(double a, double b, bool dag) {
  SOp o = sop_none();
  o.kind = SOP_BIDIAG; o.dag = dag; o.a = a; o.b = b; o.inv_a = 1.0 / a;
  sop_round(o);
  return o;
}
// (a + b S)^-1 with S^Ls = -mf: x_{last} = c0 y_{last} + sum_j w_j y_j, then recurrence
SOp sop_inv(double a, double b, bool dag, int Ls, double mf) {
  SOp o = sop_none();
  o.kind = SOP_INV; o.dag = dag; o.a = a; o.b = b; o.inv_a = 1.0 / a;
  const double rho = -b / a;
  const double c0 = 1.0 / (a * (1.0 + mf * std::pow(rho, Ls)));
  o.c0 = c0;
  double rk = rho;
  for (int j = 0; j < Ls - 1; j++) { o.w[j] = -mf * rk * c0; rk *= rho; }
  sop_round(o);
  return o;
}
SChain chain(SOp a = sop_none(), SOp b = sop_none()) {
  SChain c;
  c.op[0] = a; c.op[1] = b;
  return c;
}

struct Ops {  // operators of a context at a given quark mass
  double b5, c5, al, be, mf;
  int Ls;
  SOp D5(bool dag) const { return sop_bidiag(b5, c5, dag); }
  SOp A5(bool dag) const { return sop_bidiag(al, be, dag); }
  SOp A5inv(bool dag) const { return sop_inv(al, be, dag, Ls, mf); }
  SOp D5inv(bool dag) const { return sop_inv(b5, c5, dag, Ls, mf); }
};
Ops ops_of(const mdwf_ctx* c, double mf) {
  Ops o;
  o.b5 = c->prm.b5; o.c5 = c->prm.c5; o.al = c->alpha5; o.be = c->beta5; o.mf = mf; o.Ls = c->Ls;
  return o;
}

// ---------------------------------------------------------------- fields / workspaces
size_t half_data_bytes(const mdwf_ctx* c, int prec, int nrhs) {
  return (size_t)c->vh * prec_nc(prec) * nrhs * c->Ls * 16;
}
size_t half_norm_bytes(const mdwf_ctx* c, int prec, int nrhs) {
  return prec_norm(prec) ? (size_t)c->vh * nrhs * c->Ls * 4 : 0;
}
size_t full_bytes(const mdwf_ctx* c, int prec, int nrhs) {
  const size_t d = half_data_bytes(c, prec, nrhs), n = half_norm_bytes(c, prec, nrhs);
  return 2 * d + ((2 * n + 255) & ~(size_t)255);
}
// parity view of a full internal field
Field view(const mdwf_ctx* c, void* base, int prec, int nrhs, int parity) {
  Field f;
  const size_t d = half_data_bytes(c, prec, nrhs), n = half_norm_bytes(c, prec, nrhs);
  f.data = (char*)base + parity * d;
  f.norm = prec_norm(prec) ? (float*)((char*)base + 2 * d + parity * n) : nullptr;
  f.nrhs = nrhs; f.Ls = c->Ls; f.vh = c->vh;
  return f;
}
Field null_field() {
  Field f;
  memset(&f, 0, sizeof f);
  return f;
}

int ws_get(mdwf_ctx* c, const std::string& name, size_t bytes, void** out) {
  DevBuf& b = c->ws[name];
  if (b.p && b.bytes >= bytes) { *out = b.p; return MDWF_SUCCESS; }
  if (b.p) { cudaFree(b.p); b.p = nullptr; b.bytes = 0; }
  CK(cudaMalloc(&b.p, bytes));
  b.bytes = bytes;
  *out = b.p;
  return MDWF_SUCCESS;
}
// a half-parity workspace field
int ws_half(mdwf_ctx* c, const std::string& name, int prec, int nrhs, Field* f) {
  void* p;
  const size_t d = half_data_bytes(c, prec, nrhs), n = half_norm_bytes(c, prec, nrhs);
  CKS(ws_get(c, name + "/" + std::to_string(prec) + "/" + std::to_string(nrhs), d + n + 256, &p));
  f->data = p;
  f->norm = prec_norm(prec) ? (float*)((char*)p + ((d + 255) & ~(size_t)255)) : nullptr;
  f->nrhs = nrhs; f->Ls = c->Ls; f->vh = c->vh;
  return MDWF_SUCCESS;
}
// algorithmic bytes of one 5D site of a field in storage precision prec
double site_bytes(int prec) { return prec == F64 ? 192.0 : prec == F32 ? 96.0 : (prec == F16 || prec == I16) ? 52.0 : 48.0; }
double half_bytes(const Field& f, int prec) { return (double)f.vh * f.nrhs * f.Ls * site_bytes(prec); }
// links: 18 (or 12) reals per link, 8 links per output 4D site
double gauge_bytes(const mdwf_ctx* c, int prec) {
  return (double)c->vh * 8 * (c->prm.gauge_recon == 12 ? 12 : 18) * prec_gsize(prec);
}
size_t field_bytes_of(const Field& f, int prec) {
  return (size_t)f.vh * prec_nc(prec) * f.nrhs * f.Ls * 16;
}

// Every instantiated CG graph holds the address of c->partials as a kernel parameter, so
// the buffer is replaced only together with the graphs: a reallocation waits for the
// device, frees the old buffer and destroys every graph (they are re-captured on their
// next use, whose first block of iterations runs eagerly and sizes the buffer first).
int ensure_reduce(mdwf_ctx* c, long long blocks, int nrhs) {
  const long long groups = (blocks + RED_GROUP - 1) / RED_GROUP;
  const size_t need = (size_t)(blocks + groups) * nrhs;   // block partials, then group partials
  if (need > c->partials_n || (size_t)groups + 1 > c->counters_n) {
    const size_t n = std::max(need, 2 * c->partials_n);
    const size_t nc = std::max((size_t)groups + 1, 2 * c->counters_n);
    CK(cudaDeviceSynchronize());
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    c->graph_bytes.clear();
    if (c->partials) cudaFree(c->partials);
    if (c->counter) cudaFree(c->counter);
    c->partials = nullptr;
    c->counter = nullptr;
    c->partials_n = c->counters_n = 0;
    CK(cudaMalloc(&c->partials, n * sizeof(double)));
    c->partials_n = n;
    CK(cudaMalloc(&c->counter, nc * sizeof(unsigned)));
    CK(cudaMemset(c->counter, 0, nc * sizeof(unsigned)));
    c->counters_n = nc;
  }
  return MDWF_SUCCESS;
}

Red red_none() {
  Red r;
  memset(&r, 0, sizeof r);
  return r;
}

// ---------------------------------------------------------------- tuner
struct Snap {
  void* p;
  size_t bytes;
};

std::string key_of(const mdwf_ctx* c, const char* tag, int prec, int nrhs, const std::string& extra) {
  std::ostringstream k;
  k << tag << "|" << c->g.X << "x" << c->g.Y << "x" << c->g.Z << "x" << c->g.T << "|Ls" << c->Ls
    << "|n" << nrhs << "|p" << prec << "|" << extra;
  return k.str();
}

void save_tune(const mdwf_ctx* c) {
  if (c->tune_file.empty()) return;
  std::ofstream f(c->tune_file);
  if (!f) return;
  f << "{\n";
  size_t i = 0;
  for (auto& kv : c->tune) {
    f << "  \"" << kv.first << "\": {\"ns\": " << kv.second.ns << ", \"ms\": " << kv.second.ms << "}"
      << (++i < c->tune.size() ? "," : "") << "\n";
  }
  f << "}\n";
}

void load_tune(mdwf_ctx* c) {
  if (c->tune_file.empty()) return;
  std::ifstream f(c->tune_file);
  if (!f) return;
  std::string line;
  while (std::getline(f, line)) {
    const size_t q0 = line.find('"'), q1 = line.find('"', q0 + 1);
    const size_t n0 = line.find("\"ns\":"), m0 = line.find("\"ms\":");
    if (q0 == std::string::npos || q1 == std::string::npos || n0 == std::string::npos || m0 == std::string::npos) continue;
    TuneEntry e;
    char* end = nullptr;
    e.ns = (int)strtol(line.c_str() + n0 + 5, &end, 10);
    // corrupt entry: ignore (valid: 1..64 sites per CTA, optionally with one of the hop
    // kernels' flags 1 << 16 (occupancy-bounded build), 1 << 17 (tensor-core kernel),
    // 1 << 18 (paired-column kernel) or 1 << 19 (bulk-staged kernel); a value no candidate
    // list holds is ignored later too)
    const int ns_only = e.ns & 0xFFFF;
    const int flags = e.ns >> 16;
    if (end == line.c_str() + n0 + 5 || e.ns <= 0 || ns_only <= 0 || ns_only > 64 ||
        (flags != 0 && flags != 1 && flags != 2 && flags != 4 && flags != 8)) continue;
    e.ms = strtod(line.c_str() + m0 + 5, nullptr);
    c->tune[line.substr(q0 + 1, q1 - q0 - 1)] = e;
  }
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus s = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &s);
  return s != cudaStreamCaptureStatusNone;
}

// tuner value flags of the hop kernels (sites per CTA in the low 16 bits): the
// occupancy-bounded build of the CUDA-core kernel, the tcgen05 tensor-core kernel, the
// paired-column CUDA-core kernel, and the bulk-staged CUDA-core kernel
constexpr int kOccBit = 1 << 16;
constexpr int kTcBit = 1 << 17;
constexpr int kPairBit = 1 << 18;
constexpr int kBulkBit = 1 << 19;

// Pick sites-per-CTA for `key` by brute force over `cands`, timing each with events.
// In-place outputs listed in `snaps` are saved before and restored after every trial run,
// so tuning does not change the result of the call.
// MDWF_FORCE_NS pins the tuner value (sites per CTA, optionally with a kernel flag) where a
// candidate list holds it; tests use it to exercise ragged last tiles and every kernel
bool forced_cfg(const std::vector<int>& cands, int* out) {
  const char* fns = getenv("MDWF_FORCE_NS");
  if (!fns) return false;
  const int f = atoi(fns);
  for (int v : {f, f | kTcBit})
    if (std::find(cands.begin(), cands.end(), v) != cands.end()) { *out = v; return true; }
  return false;
}

template <typename F>
int tuned_ns(mdwf_ctx* c, const std::string& key, const std::vector<int>& cands, int dflt,
             const std::vector<Snap>& snaps, cudaStream_t st, F run, int* ns_out) {
  if (forced_cfg(cands, ns_out)) return MDWF_SUCCESS;
  auto it = c->tune.find(key);
  if (it != c->tune.end()) {
    if (std::find(cands.begin(), cands.end(), it->second.ns) != cands.end()) {
      *ns_out = it->second.ns;
      return MDWF_SUCCESS;
    }
  }
  if (!c->tuning || cands.size() <= 1 || capturing(st)) {
    *ns_out = dflt;
    return MDWF_SUCCESS;
  }
  std::vector<void*> saved(snaps.size(), nullptr);
  for (size_t i = 0; i < snaps.size(); i++) {
    CK(cudaMalloc(&saved[i], snaps[i].bytes));
    CK(cudaMemcpyAsync(saved[i], snaps[i].p, snaps[i].bytes, cudaMemcpyDeviceToDevice, st));
  }
  auto restore = [&]() -> int {
    for (size_t i = 0; i < snaps.size(); i++)
      CK(cudaMemcpyAsync(snaps[i].p, saved[i], snaps[i].bytes, cudaMemcpyDeviceToDevice, st));
    return MDWF_SUCCESS;
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = dflt;
  double best_ms = 1e30;
  for (int ns : cands) {
    double tmin = 1e30;
    for (int rep = 0; rep < 3; rep++) {
      CKS(restore());
      CK(cudaEventRecord(e0, st));
      CKS(run(ns));
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) tmin = std::min(tmin, (double)ms);
    }
    if (tmin < best_ms) { best_ms = tmin; best = ns; }
  }
  CKS(restore());
  CK(cudaStreamSynchronize(st));
  for (void* p : saved) cudaFree(p);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tune[key] = TuneEntry{best, best_ms};
  save_tune(c);
  *ns_out = best;
  return MDWF_SUCCESS;
}


// sites per CTA: powers of two, plus for the hop kernels (dense = true) every size up to
// the thread limit (the wave count over 152 SMs matters as much as occupancy)
std::vector<int> ns_candidates(int W, int maxthreads = MAXTHREADS, bool dense = false) {
  std::vector<int> v;
  for (int ns = 1; ns <= 64; ns++) {
    if (ns * W > maxthreads) break;
    if (dense || (ns & (ns - 1)) == 0) v.push_back(ns);
  }
  if (v.empty()) v.push_back(1);
  return v;
}
int ns_default(int W) {
  int ns = 1;
  while (2 * ns * W <= 128) ns *= 2;
  return ns;
}

// ---------------------------------------------------------------- gauge
int gauge_for(mdwf_ctx* c, int prec, const void** out) {
  if (!c->gauge_loaded) { g_last_error = "no gauge field loaded"; return MDWF_ERR_STATE; }
  if (!c->gauge[prec][0]) {
    const int r = c->prm.gauge_recon;
    const int gs = gauge_stride(prec, r);
    const long long nl = c->vh * 8;
    for (int par = 0; par < 2; par++) {
      CK(cudaMalloc(&c->gauge[prec][par], nl * gs * prec_gsize(prec)));
      CK(launch_gauge_convert(prec, (const double*)c->gauge[F64][par], c->gauge[prec][par], nl,
                              c->gs[F64], gs, r == 12 ? 12 : 18, 0));
      c->launches++;
    }
    CK(cudaDeviceSynchronize());
    c->gs[prec] = gs;
  }
  *out = nullptr;
  return MDWF_SUCCESS;
}

// ---------------------------------------------------------------- hop launcher
struct Epi {
  bool on = false;
  SChain post = chain();
  double hc = 1.0;
  Field center = null_field();
  SChain cop = chain();
  double cc = 1.0;
  bool norm_pre = false;
  SChain fin = chain();
  Field raxpy = null_field();
  double mf = 0.0;
};

std::string chain_sig(const SChain& ch) {
  std::string s;
  for (int i = 0; i < 2; i++) s += std::to_string(ch.op[i].kind) + (ch.op[i].dag ? "d" : "");
  return s;
}

// bytes of one face: 12 compute-type reals per face site and column, then (F16, int16) a
// scale
size_t face_bytes_of(const mdwf_ctx* c, int prec, int nrhs) {
  const size_t W = (size_t)nrhs * c->Ls;
  const size_t data = (size_t)c->slice_vh * W * 12 * (prec == F64 ? 8 : 4);
  return ((data + 255) & ~(size_t)255) + (prec == F16 || prec == I16 ? (size_t)c->slice_vh * W * 4 : 0);
}

// One hop on a T-partitioned lattice: pack the input half's two faces, launch the interior
// timeslices, exchange, launch the first and last timeslices with their t neighbours
// across the boundary taken from the received faces (bit-identical to one launch on the
// undecomposed lattice: every site runs the same code on the same reals).
int hop_partitioned(mdwf_ctx* c, int prec, bool dag, bool r12, bool epi, const HopParams& p, int cfg,
                    const Field& in, const Field& out, cudaStream_t st) {
  if (!c->xfn) { g_last_error = "T-partitioned context without a face exchange"; return MDWF_ERR_STATE; }
  const long long sv = c->slice_vh, vh = c->vh;
  const size_t fb = face_bytes_of(c, prec, in.nrhs);
  const size_t fdata = (size_t)sv * in.nrhs * c->Ls * 12 * (prec == F64 ? 8 : 4);
  void* buf[4];
  if (c->user_faces[0] && c->user_face_bytes >= fb) {
    for (int k = 0; k < 4; k++) buf[k] = c->user_faces[k];
  } else {
    const char* names[4] = {"face_send_lo", "face_send_hi", "face_recv_lo", "face_recv_hi"};
    for (int k = 0; k < 4; k++) CKS(ws_get(c, names[k], fb, &buf[k]));
  }
  auto norm_of = [&](void* b) -> float* {
    return prec == F16 || prec == I16 ? (float*)((char*)b + ((fdata + 255) & ~(size_t)255)) : nullptr;
  };
  const int SF = dag ? -1 : 1;
  FaceParams fp;
  fp.in = in; fp.slice_vh = sv;
  fp.first = 0; fp.face = buf[0]; fp.norm = norm_of(buf[0]);      // first timeslice, for the hop t+1 below
  CK(launch_pack_face(prec, SF, fp, st));
  fp.first = vh - sv; fp.face = buf[1]; fp.norm = norm_of(buf[1]); // last timeslice, for the hop t-1 above
  CK(launch_pack_face(prec, -SF, fp, st));
  c->launches += 2;
  c->bytes += 2.0 * half_bytes(in, prec) / (double)c->g.T + 2.0 * fb;
  const bool tc = (cfg & kTcBit) != 0;
  auto launch = [&](long long x0, long long x1, int mode, void* face, long long base) -> int {
    if (x1 <= x0) return MDWF_SUCCESS;
    HopParams q = p;
    q.ns = cfg & 0xFFFF;
    q.status = c->dev_status;
    q.x_begin = x0; q.x_end = x1;
    q.face_mode = mode; q.face = face; q.face_norm = face ? norm_of(face) : nullptr; q.face_base = base;
    cudaError_t err = tc ? launch_hop_tc(prec, dag, r12, epi, q, st)
                         : launch_hop(prec, dag, r12, epi, (cfg & kOccBit) != 0, (cfg & kPairBit) != 0, false,
                                      (cfg & kBulkBit) != 0, q, st);
    c->launches++;
    if (err != cudaSuccess) { set_err("launch_hop", err); return MDWF_ERR_CUDA; }
    return MDWF_SUCCESS;
  };
  CKS(launch(sv, vh - sv, 0, nullptr, 0));                 // interior, while the faces travel
  const int xs = c->xfn(c->xuser, buf[0], buf[1], buf[2], buf[3], fb, (void*)st);
  if (xs != 0) {
    if (g_last_error.empty()) g_last_error = "face exchange failed";
    return xs < 0 ? xs : MDWF_ERR_CUDA;
  }
  CKS(launch(0, sv, 1, buf[2], vh - sv));                   // first timeslice: t-1 from below
  CKS(launch(vh - sv, vh, 2, buf[3], 0));                   // last timeslice: t+1 from above
  c->bytes += half_bytes(in, prec) + gauge_bytes(c, prec) + (p.has_center ? half_bytes(p.center, prec) : 0.0) +
              (p.axpy_r ? 2.0 * half_bytes(p.raxpy, prec) : half_bytes(out, prec));
  return MDWF_SUCCESS;
}

int hop(mdwf_ctx* c, int prec, bool dag, const Field& in, const Field& out, int pout, const Epi& e,
        Red red, cudaStream_t st, std::vector<Snap> snaps = {}) {
  const void* unused;
  CKS(gauge_for(c, prec, &unused));
  HopParams p;
  memset(&p, 0, sizeof p);
  p.gauge = c->gauge[prec][pout];
  p.gs = c->gs[prec];
  p.in = in; p.out = out; p.pout = pout; p.g = c->g; p.t_bc = c->prm.t_bc;
  p.mf = e.mf;
  p.post = e.post; p.hc = e.hc;
  p.has_center = e.center.data != nullptr;
  p.center = e.center; p.cop = e.cop; p.cc = e.cc;
  // the epilogue applies the centre's operator per site from s +- 1: one bidiagonal op at most
  if (e.cop.op[1].kind != SOP_NONE || e.cop.op[0].kind == SOP_INV) {
    g_last_error = "internal: centre operator must be empty or one bidiagonal op";
    return MDWF_ERR_ARG;
  }
  p.norm_pre = e.norm_pre; p.fin = e.fin;
  p.axpy_r = e.raxpy.data != nullptr;
  p.raxpy = e.raxpy;
  p.red = red;
  const bool r12 = c->prm.gauge_recon == 12;
  const int W = in.nrhs * in.Ls;
  // F16 / BF16: the tcgen05 tensor-core kernel (tuner value | kTcBit, sites per CTA in the
  // low bits) competes with the CUDA-core kernel; MDWF_TC=0 leaves it out, MDWF_TC=1 uses
  // it alone
  const char* use_tc = getenv("MDWF_TC");
  const bool tc_ok = hop_tc_supported(prec, p, r12) && !(use_tc && use_tc[0] == '0');
  const bool tc_only = tc_ok && use_tc && use_tc[0] == '1';
  std::vector<int> cands;
  if (!tc_only) {
    for (int ns : ns_candidates(W, MAXTHREADS, true)) {
      HopParams q = p;
      q.ns = ns;
      if (hop_smem_bytes(prec, q, e.on) > 200 * 1024) continue;
      cands.push_back(ns);
      // fused 32-bit kernels also come in an occupancy-bounded build (tuner value | kOccBit)
      if (e.on && prec != F64) cands.push_back(ns | kOccBit);
    }
    // the paired-column kernel: two columns per thread, ns * W / 2 threads
    HopParams q = p;
    q.ns = 1;
    if (hop_pair_supported(prec, q)) {
      for (int ns = 1; ns <= 64 && ns * W / 2 <= MAXTHREADS; ns++) {
        q.ns = ns;
        if (hop_smem_bytes(prec, q, e.on, true) > 200 * 1024) continue;
        cands.push_back(ns | kPairBit);
      }
    }
    // the bulk-staged kernel (undecomposed lattices: a partition's face timeslices take
    // their t neighbours from the faces)
    if (hop_bulk_supported(prec, q) && c->prm.t_ranks == 1) {
      for (int ns : ns_candidates(W, MAXTHREADS, true)) {
        q.ns = ns;
        if (hop_smem_bytes(prec, q, e.on, false, true) > 200 * 1024) continue;
        cands.push_back(ns | kBulkBit);
      }
    }
  }
  if (tc_ok) {
    for (int ns = 1; ns <= 16; ns *= 2) {
      HopParams q = p;
      q.ns = ns;
      if (hop_tc_smem_bytes(q) > 200 * 1024 || hop_tc_tmem_cols(q) > 256) break;
      cands.push_back(ns | kTcBit);
    }
  }
  if (cands.empty()) { g_last_error = "hop: shared memory"; return MDWF_ERR_ARG; }
  int dflt = cands.front();
  if (tc_only) {
    dflt = cands.back();
    for (int v : cands) if ((v & 0xFFFF) == 4) dflt = v;
  } else {
    const int want = std::min(ns_default(W), cands.back() & 0xFFFF);
    for (int v : cands) if (v == want) dflt = v;
  }
  const bool emu = prec == F64 && c->emu_active;
  const std::string key = key_of(c, dag ? "hopdag" : "hop", prec, in.nrhs,
                                 std::string(tc_only ? "tc" : "") + (emu ? "emu" : "") + (e.on ? "epi" : "plain") + chain_sig(e.post) +
                                     chain_sig(e.fin) + (p.has_center ? "c" : "") + (p.axpy_r ? "a" : "") +
                                     (red.mode ? "r" : ""));
  p.x_begin = 0;
  p.x_end = c->vh;
  p.bc_lo = c->prm.t_rank == 0;
  p.bc_hi = c->prm.t_rank == c->prm.t_ranks - 1;
  if (c->prm.t_ranks > 1) {
    if (red.mode != RED_NONE) {
      g_last_error = "a reduction over a T-partitioned lattice needs a global sum";
      return MDWF_ERR_STATE;
    }
    int cfg = dflt;
    auto it = c->tune.find(key);
    if (!forced_cfg(cands, &cfg) && it != c->tune.end() &&
        std::find(cands.begin(), cands.end(), it->second.ns) != cands.end())
      cfg = it->second.ns;
    return hop_partitioned(c, prec, dag, r12, e.on, p, cfg, in, out, st);
  }
  auto run = [&](int cfg) -> int {
    HopParams q = p;
    const int ns = cfg & 0xFFFF;
    const bool tc = (cfg & kTcBit) != 0;
    q.ns = ns;
    q.status = c->dev_status;
    const long long blocks = (c->vh + ns - 1) / ns;
    if (q.red.mode != RED_NONE) {
      CKS(ensure_reduce(c, blocks, in.nrhs));
      q.red.partials = c->partials;
      q.red.counter = c->counter;
    }
    cudaError_t err = tc ? launch_hop_tc(prec, dag, r12, e.on, q, st)
                         : launch_hop(prec, dag, r12, e.on, (cfg & kOccBit) != 0, (cfg & kPairBit) != 0, emu,
                                      (cfg & kBulkBit) != 0, q, st);
    c->launches++;
    c->bytes += half_bytes(in, prec) + gauge_bytes(c, prec) + (q.has_center ? half_bytes(e.center, prec) : 0.0) +
                (q.axpy_r ? 2.0 * half_bytes(e.raxpy, prec) : half_bytes(out, prec));
    if (err != cudaSuccess) { set_err("launch_hop", err); return MDWF_ERR_CUDA; }
    return MDWF_SUCCESS;
  };
  if (red.mode == RED_CG_BETA || red.mode == RED_CG_ALPHA)
    snaps.push_back(Snap{c->cg, 64 * sizeof(CGScalars)});
  if (p.axpy_r) {
    snaps.push_back(Snap{e.raxpy.data, field_bytes_of(e.raxpy, prec)});
    if (e.raxpy.norm) snaps.push_back(Snap{e.raxpy.norm, (size_t)e.raxpy.vh * e.raxpy.nrhs * e.raxpy.Ls * 4});
  }
  int ns;
  CKS(tuned_ns(c, key, cands, dflt, snaps, st, run, &ns));
  return run(ns);
}

// s-local launches
int sl_chain(mdwf_ctx* c, int prec, const Field& out, const Field& in, const SChain& ch, double ca,
             const Field* add, double cb, double mf, cudaStream_t st) {
  SLParams p;
  memset(&p, 0, sizeof p);
  p.a = out; p.b = in; p.c = add ? *add : null_field(); p.vh = c->vh;
  p.chain = ch; p.ca = ca; p.cb = cb; p.mf = mf; p.red = red_none();
  const int W = in.nrhs * in.Ls;
  auto run = [&](int ns) -> int {
    SLParams q = p;
    q.ns = ns;
    cudaError_t err = launch_chain(prec, q, st);
    c->launches++;
    c->bytes += half_bytes(in, prec) * (add ? 3.0 : 2.0);
    if (err != cudaSuccess) { set_err("launch_chain", err); return MDWF_ERR_CUDA; }
    return MDWF_SUCCESS;
  };
  int ns;
  CKS(tuned_ns(c, key_of(c, "chain", prec, in.nrhs, chain_sig(ch) + (add ? "a" : "")), ns_candidates(W),
               ns_default(W), {}, st, run, &ns));
  return run(ns);
}

// a = ca*b + cb*c with optional |a|^2 -> reduce mode
int sl_axpby(mdwf_ctx* c, int prec, const Field* a, const Field& b, double ca, const Field* cfield, double cb,
             Red red, cudaStream_t st) {
  SLParams p;
  memset(&p, 0, sizeof p);
  p.a = a ? *a : null_field(); p.b = b; p.c = cfield ? *cfield : null_field();
  p.vh = c->vh; p.ca = ca; p.cb = cb; p.red = red;
  const int W = b.nrhs * b.Ls;
  const int ns = ns_default(W);
  p.ns = ns;
  const long long blocks = (c->vh + ns - 1) / ns;
  if (red.mode != RED_NONE) {
    CKS(ensure_reduce(c, blocks, b.nrhs));
    p.red.partials = c->partials;
    p.red.counter = c->counter;
  }
  cudaError_t err = launch_axpby(prec, p, st);
  c->launches++;
  c->bytes += half_bytes(b, prec) * (1.0 + (cfield ? 1.0 : 0.0) + (a ? 1.0 : 0.0));
  if (err != cudaSuccess) { set_err("launch_axpby", err); return MDWF_ERR_CUDA; }
  return MDWF_SUCCESS;
}

int sl_convert(mdwf_ctx* c, int po, const Field& out, int pi, const Field& in, bool accumulate, bool zero_in,
               cudaStream_t st) {
  SLParams p;
  memset(&p, 0, sizeof p);
  p.a = out; p.b = in; p.vh = c->vh; p.ca = accumulate ? 1.0 : 0.0; p.cb = zero_in ? 1.0 : 0.0;
  const int W = in.nrhs * in.Ls;
  p.ns = ns_default(W);
  cudaError_t err = launch_convert(po, pi, p, st);
  c->launches++;
  c->bytes += half_bytes(in, pi) * (zero_in ? 2.0 : 1.0) + half_bytes(out, po) * (accumulate ? 2.0 : 1.0);
  if (err != cudaSuccess) { set_err("launch_convert", err); return MDWF_ERR_CUDA; }
  return MDWF_SUCCESS;
}

// per-rhs Re <a, b> into host vector
int dot(mdwf_ctx* c, int prec, const Field& a, const Field& b, std::vector<double>& out, cudaStream_t st);
int rhs_axpy(mdwf_ctx* c, int prec, const Field& a, const Field& b, const std::vector<double>& coef, cudaStream_t st);

Red red_store(mdwf_ctx* c, int nrhs) {
  Red r = red_none();
  r.mode = RED_STORE; r.counter = c->counter; r.out = c->red_out; r.nrhs = nrhs;
  return r;
}
Red red_cg(mdwf_ctx* c, int mode, int nrhs) {
  Red r = red_none();
  r.mode = mode; r.counter = c->counter; r.cg = c->cg; r.nrhs = nrhs;
  return r;
}

// per-rhs |f|^2 into host vector
int norm2(mdwf_ctx* c, int prec, const Field& f, std::vector<double>& out, cudaStream_t st) {
  CKS(sl_axpby(c, prec, nullptr, f, 1.0, nullptr, 0.0, red_store(c, f.nrhs), st));
  CK(cudaMemcpyAsync(c->red_host, c->red_out, f.nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  out.assign(c->red_host, c->red_host + f.nrhs);
  return MDWF_SUCCESS;
}

int dot(mdwf_ctx* c, int prec, const Field& a, const Field& b, std::vector<double>& out, cudaStream_t st) {
  SLParams p;
  memset(&p, 0, sizeof p);
  p.b = a; p.c = b; p.vh = c->vh; p.red = red_store(c, a.nrhs);
  const int W = a.nrhs * a.Ls;
  p.ns = ns_default(W);
  CKS(ensure_reduce(c, (c->vh + p.ns - 1) / p.ns, a.nrhs));
  p.red.partials = c->partials;
  p.red.counter = c->counter;
  cudaError_t err = launch_dot(prec, p, st);
  c->launches++;
  c->bytes += 2.0 * half_bytes(a, prec);
  if (err != cudaSuccess) { set_err("launch_dot", err); return MDWF_ERR_CUDA; }
  CK(cudaMemcpyAsync(c->red_host, c->red_out, a.nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  out.assign(c->red_host, c->red_host + a.nrhs);
  return MDWF_SUCCESS;
}

int rhs_axpy(mdwf_ctx* c, int prec, const Field& a, const Field& b, const std::vector<double>& coef, cudaStream_t st) {
  for (size_t i = 0; i < coef.size(); i++) c->red_host[i] = coef[i];
  CK(cudaMemcpyAsync(c->red_out, c->red_host, coef.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  SLParams p;
  memset(&p, 0, sizeof p);
  p.a = a; p.b = b; p.vh = c->vh; p.red = red_store(c, a.nrhs);
  p.ns = ns_default(a.nrhs * a.Ls);
  cudaError_t err = launch_rhs_axpy(prec, p, st);
  c->launches++;
  c->bytes += 3.0 * half_bytes(a, prec);
  if (err != cudaSuccess) { set_err("launch_rhs_axpy", err); return MDWF_ERR_CUDA; }
  CK(cudaStreamSynchronize(st));
  return MDWF_SUCCESS;
}

// ---------------------------------------------------------------- operator compositions
// M_pc in (odd) -> out (odd).   tmp fields from the workspace.
int apply_mpc(mdwf_ctx* c, int prec, const Field& in, const Field& out, cudaStream_t st) {
  const Ops o = ops_of(c, c->prm.mf);
  Field t, w;
  CKS(ws_half(c, "mpc_t", prec, in.nrhs, &t));
  CKS(ws_half(c, "mpc_w", prec, in.nrhs, &w));
  CKS(sl_chain(c, prec, t, in, chain(o.D5(false)), 1.0, nullptr, 0.0, o.mf, st));
  Epi e1;
  e1.on = true; e1.post = chain(o.A5inv(false), o.D5(false)); e1.mf = o.mf;
  CKS(hop(c, prec, false, t, w, 0, e1, red_none(), st));
  Epi e2;
  e2.on = true; e2.post = chain(o.A5inv(false)); e2.hc = -0.25; e2.center = in; e2.mf = o.mf;
  return hop(c, prec, false, w, out, 1, e2, red_none(), st);
}

int apply_mpc_dag(mdwf_ctx* c, int prec, const Field& in, const Field& out, cudaStream_t st) {
  const Ops o = ops_of(c, c->prm.mf);
  Field qt, y;
  CKS(ws_half(c, "mpcd_q", prec, in.nrhs, &qt));
  CKS(ws_half(c, "mpcd_y", prec, in.nrhs, &y));
  CKS(sl_chain(c, prec, qt, in, chain(o.A5inv(true)), 1.0, nullptr, 0.0, o.mf, st));
  Epi e3;
  e3.on = true; e3.post = chain(o.D5(true), o.A5inv(true)); e3.mf = o.mf;
  CKS(hop(c, prec, true, qt, y, 0, e3, red_none(), st));
  Epi e4;
  e4.on = true; e4.post = chain(o.D5(true)); e4.hc = -0.25; e4.center = qt; e4.cop = chain(o.A5(true));
  e4.mf = o.mf;
  return hop(c, prec, true, y, out, 1, e4, red_none(), st);
}

// M_sym in (odd) -> out (odd): M_sym = 1 - (1/4) X H_oe X H_eo, X = D5 A5^-1 (two fused
// hop kernels, no input pre-chain)
int apply_mpc_sym(mdwf_ctx* c, int prec, const Field& in, const Field& out, cudaStream_t st) {
  const Ops o = ops_of(c, c->prm.mf);
  Field w;
  CKS(ws_half(c, "mpc_w", prec, in.nrhs, &w));
  Epi e1;
  e1.on = true; e1.post = chain(o.A5inv(false), o.D5(false)); e1.mf = o.mf;
  CKS(hop(c, prec, false, in, w, 0, e1, red_none(), st));
  Epi e2;
  e2.on = true; e2.post = chain(o.A5inv(false), o.D5(false)); e2.hc = -0.25; e2.center = in; e2.mf = o.mf;
  return hop(c, prec, false, w, out, 1, e2, red_none(), st);
}

// M_sym^+ = 1 - (1/4) (H^+)_oe X^+ (H^+)_eo X^+, X^+ = A5^-+ D5^+
int apply_mpc_sym_dag(mdwf_ctx* c, int prec, const Field& in, const Field& out, cudaStream_t st) {
  const Ops o = ops_of(c, c->prm.mf);
  Field qt, y;
  CKS(ws_half(c, "mpcd_q", prec, in.nrhs, &qt));
  CKS(ws_half(c, "mpcd_y", prec, in.nrhs, &y));
  CKS(sl_chain(c, prec, qt, in, chain(o.D5(true), o.A5inv(true)), 1.0, nullptr, 0.0, o.mf, st));
  Epi e3;
  e3.on = true; e3.post = chain(o.D5(true), o.A5inv(true)); e3.mf = o.mf;
  CKS(hop(c, prec, true, qt, y, 0, e3, red_none(), st));
  Epi e4;
  e4.on = true; e4.hc = -0.25; e4.center = in; e4.mf = o.mf;
  return hop(c, prec, true, y, out, 1, e4, red_none(), st);
}

// the odd-site operator of a preconditioned form and its adjoint
int apply_M(mdwf_ctx* c, int form, int prec, const Field& in, const Field& out, cudaStream_t st) {
  return form == MDWF_PC_SYM ? apply_mpc_sym(c, prec, in, out, st) : apply_mpc(c, prec, in, out, st);
}
int apply_Mdag(mdwf_ctx* c, int form, int prec, const Field& in, const Field& out, cudaStream_t st) {
  return form == MDWF_PC_SYM ? apply_mpc_sym_dag(c, prec, in, out, st) : apply_mpc_dag(c, prec, in, out, st);
}

// full 5D D (or D^+) on both parities at quark mass mf
int apply_full(mdwf_ctx* c, int prec, bool dag, const Field in[2], const Field out[2], double mf, cudaStream_t st) {
  const Ops o = ops_of(c, mf);
  if (!dag) {
    Field t[2];
    CKS(ws_half(c, "full_t0", prec, in[0].nrhs, &t[0]));
    CKS(ws_half(c, "full_t1", prec, in[0].nrhs, &t[1]));
    for (int par = 0; par < 2; par++) CKS(sl_chain(c, prec, t[par], in[par], chain(o.D5(false)), 1.0, nullptr, 0.0, mf, st));
    for (int par = 0; par < 2; par++) {
      Epi e;
      e.on = true; e.hc = -0.5; e.center = in[par]; e.cop = chain(o.A5(false)); e.mf = mf;
      CKS(hop(c, prec, false, t[1 - par], out[par], par, e, red_none(), st));
    }
  } else {
    for (int par = 0; par < 2; par++) {
      Epi e;
      e.on = true; e.post = chain(o.D5(true)); e.hc = -0.5; e.center = in[par]; e.cop = chain(o.A5(true)); e.mf = mf;
      CKS(hop(c, prec, true, in[1 - par], out[par], par, e, red_none(), st));
    }
  }
  return MDWF_SUCCESS;
}

// ---------------------------------------------------------------- CG
struct CGSet {
  int prec, prec_x, nrhs, form;
  Field x, r, p, ph, w, qt, y;
};

int make_cgset(mdwf_ctx* c, int prec, int prec_x, int nrhs, int form, CGSet* s) {
  s->prec = prec; s->prec_x = prec_x; s->nrhs = nrhs; s->form = form;
  CKS(ws_half(c, "cg_x", prec_x, nrhs, &s->x));
  CKS(ws_half(c, "cg_r", prec, nrhs, &s->r));
  CKS(ws_half(c, "cg_p", prec, nrhs, &s->p));
  CKS(ws_half(c, "cg_ph", prec, nrhs, &s->ph));
  CKS(ws_half(c, "cg_w", prec, nrhs, &s->w));
  CKS(ws_half(c, "cg_qt", prec, nrhs, &s->qt));
  CKS(ws_half(c, "cg_y", prec, nrhs, &s->y));
  return MDWF_SUCCESS;
}

int cg_update(mdwf_ctx* c, const CGSet& v, const SChain& ch, bool phat, cudaStream_t st);

// One CG iteration on M_sym^+ M_sym (X = D5 A5^-1): K1 w_e = X H_eo p; K2 q = p - X H_oe w / 4
// with |q|^2 -> alpha; X^+ q (s-local); K3 y_e = X^+ (H^+)_eo X^+ q; K4 r -= alpha
// (q - (H^+)_oe y / 4) with |r|^2 -> beta; then x += alpha p, p = r + beta p.
int cg_iteration_sym(mdwf_ctx* c, const CGSet& v, cudaStream_t st) {
  const Ops o = ops_of(c, c->prm.mf);
  const int P = v.prec;
  Epi e1;
  e1.on = true; e1.post = chain(o.A5inv(false), o.D5(false)); e1.mf = o.mf;
  CKS(hop(c, P, false, v.p, v.w, 0, e1, red_none(), st));
  Epi e2;
  e2.on = true; e2.post = chain(o.A5inv(false), o.D5(false)); e2.hc = -0.25; e2.center = v.p; e2.norm_pre = true;
  e2.mf = o.mf;
  CKS(hop(c, P, false, v.w, v.qt, 1, e2, red_cg(c, RED_CG_ALPHA, v.nrhs), st));
  CKS(sl_chain(c, P, v.ph, v.qt, chain(o.D5(true), o.A5inv(true)), 1.0, nullptr, 0.0, o.mf, st));
  Epi e3;
  e3.on = true; e3.post = chain(o.D5(true), o.A5inv(true)); e3.mf = o.mf;
  CKS(hop(c, P, true, v.ph, v.y, 0, e3, red_none(), st));
  Epi e4;
  e4.on = true; e4.hc = -0.25; e4.center = v.qt; e4.raxpy = v.r; e4.mf = o.mf;
  CKS(hop(c, P, true, v.y, v.r, 1, e4, red_cg(c, RED_CG_BETA, v.nrhs), st));
  return cg_update(c, v, chain(), false, st);
}

// One CG iteration on M_pc^+ M_pc: five kernels, scalars stay on the device.
int cg_iteration(mdwf_ctx* c, const CGSet& v, cudaStream_t st) {
  if (v.form == MDWF_PC_SYM) return cg_iteration_sym(c, v, st);
  const Ops o = ops_of(c, c->prm.mf);
  const int P = v.prec;
  Epi e1;  // w_e = D5 A5^-1 H_eo phat
  e1.on = true; e1.post = chain(o.A5inv(false), o.D5(false)); e1.mf = o.mf;
  CKS(hop(c, P, false, v.ph, v.w, 0, e1, red_none(), st));
  Epi e2;  // q = p - A5^-1 H_oe w / 4 ; |q|^2 -> alpha ; store qt = A5^-+ q
  e2.on = true; e2.post = chain(o.A5inv(false)); e2.hc = -0.25; e2.center = v.p; e2.norm_pre = true;
  e2.fin = chain(o.A5inv(true)); e2.mf = o.mf;
  CKS(hop(c, P, false, v.w, v.qt, 1, e2, red_cg(c, RED_CG_ALPHA, v.nrhs), st));
  Epi e3;  // y_e = A5^-+ D5^+ H_oe^+ qt
  e3.on = true; e3.post = chain(o.D5(true), o.A5inv(true)); e3.mf = o.mf;
  CKS(hop(c, P, true, v.qt, v.y, 0, e3, red_none(), st));
  Epi e4;  // s = A5^+ qt - D5^+ H_eo^+ y / 4 ; r -= alpha s ; |r|^2 -> beta
  e4.on = true; e4.post = chain(o.D5(true)); e4.hc = -0.25; e4.center = v.qt; e4.cop = chain(o.A5(true));
  e4.raxpy = v.r; e4.mf = o.mf;
  CKS(hop(c, P, true, v.y, v.r, 1, e4, red_cg(c, RED_CG_BETA, v.nrhs), st));
  return cg_update(c, v, chain(o.D5(false)), true, st);
}

// x += alpha p ; p = r + beta p ; phat = ch(p) when phat
int cg_update(mdwf_ctx* c, const CGSet& v, const SChain& ch, bool phat, cudaStream_t st) {
  const Ops o = ops_of(c, c->prm.mf);
  const int P = v.prec;
  SLParams q;
  memset(&q, 0, sizeof q);
  q.a = v.p; q.b = v.r; q.c = phat ? v.ph : null_field(); q.x = v.x; q.vh = c->vh; q.chain = ch; q.mf = o.mf;
  q.red = red_cg(c, RED_NONE, v.nrhs);
  const int W = v.nrhs * c->Ls;
  std::vector<Snap> snaps = {{v.x.data, field_bytes_of(v.x, v.prec_x)}, {v.p.data, field_bytes_of(v.p, P)}};
  if (v.x.norm) snaps.push_back({v.x.norm, (size_t)c->vh * W * 4});
  if (v.p.norm) snaps.push_back({v.p.norm, (size_t)c->vh * W * 4});
  auto run = [&](int ns) -> int {
    SLParams qq = q;
    qq.ns = ns;
    cudaError_t err = launch_cg_update(v.prec_x, P, qq, st);
    c->launches++;
    c->bytes += 2.0 * half_bytes(v.x, v.prec_x) + (phat ? 4.0 : 3.0) * half_bytes(v.p, P);
    if (err != cudaSuccess) { set_err("launch_cg_update", err); return MDWF_ERR_CUDA; }
    return MDWF_SUCCESS;
  };
  int ns;
  CKS(tuned_ns(c, key_of(c, "cgupd", P, v.nrhs, std::to_string(v.prec_x) + (phat ? "" : "n")), ns_candidates(W),
               ns_default(W), snaps, st, run, &ns));
  return run(ns);
}

// the device status flag (a kernel whose bounded wait gave up) -> MDWF_ERR_TIMEOUT
int check_status(mdwf_ctx* c, cudaStream_t st) {
  CK(cudaMemcpyAsync(c->status_host, c->dev_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*c->status_host) {
    CK(cudaMemsetAsync(c->dev_status, 0, sizeof(int), st));
    g_last_error = "a tensor-core hop kernel gave up waiting for its matrix products";
    return MDWF_ERR_TIMEOUT;
  }
  return MDWF_SUCCESS;
}

int pull_scalars(mdwf_ctx* c, int nrhs, cudaStream_t st) {
  CK(cudaMemcpyAsync(c->cg_host, c->cg, nrhs * sizeof(CGScalars), cudaMemcpyDeviceToHost, st));
  return check_status(c, st);
}
int push_scalars(mdwf_ctx* c, int nrhs, cudaStream_t st) {
  CK(cudaMemcpyAsync(c->cg, c->cg_host, nrhs * sizeof(CGScalars), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return MDWF_SUCCESS;
}

// run n iterations, as a CUDA graph when asked (captured once per shape and buffer set)
int run_iterations(mdwf_ctx* c, const CGSet& v, int n, bool use_graph, cudaStream_t st) {
  if (!use_graph || st == 0) {
    for (int i = 0; i < n; i++) CKS(cg_iteration(c, v, st));
    return MDWF_SUCCESS;
  }
  char key[256];
  snprintf(key, sizeof key, "%d/%d/%d/%d/%d/%p/%p/%p", v.prec, v.prec_x, v.nrhs, v.form, n, v.r.data, v.x.data,
           (void*)st);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int s = MDWF_SUCCESS;
    const long long before = c->launches;
    const double bytes_before = c->bytes;
    for (int i = 0; i < n && s == MDWF_SUCCESS; i++) s = cg_iteration(c, v, st);
    c->graph_bytes[key] = c->bytes - bytes_before;
    c->bytes = bytes_before;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s != MDWF_SUCCESS) return s;
    CK(e);
    cudaGraphExec_t exec;
    CK(cudaGraphInstantiate(&exec, graph, 0));
    cudaGraphDestroy(graph);
    c->launches = before;  // captured launches are counted at replay
    it = c->graphs.emplace(key, exec).first;
  }
  CK(cudaGraphLaunch(it->second, st));
  c->launches += (v.form == MDWF_PC_SYM ? 6LL : 5LL) * n;
  c->bytes += c->graph_bytes[key];
  return MDWF_SUCCESS;
}

struct SolveState {
  int nrhs;
  std::vector<double> bnorm2;     // |b~|^2
  std::vector<double> true_rel;   // last true relative residual
  std::vector<int> done;
  std::vector<int> iters;
  int ru = 0;
  int fp64_res = 0;               // FP64 recomputations of b~ - M x
  int emu_res = 0;                // ... of which in emulated FP64
};

// res = b~ - M x (FP64), |res|^2 per rhs
int true_residual(mdwf_ctx* c, int form, const Field& bt, const Field& x, const Field& res, std::vector<double>& r2,
                  cudaStream_t st) {
  Field q;
  CKS(ws_half(c, "tr_q", F64, x.nrhs, &q));
  CKS(apply_M(c, form, F64, x, q, st));
  CKS(sl_axpby(c, F64, &res, bt, 1.0, &q, -1.0, red_store(c, x.nrhs), st));
  CK(cudaMemcpyAsync(c->red_host, c->red_out, x.nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  r2.assign(c->red_host, c->red_host + x.nrhs);
  return MDWF_SUCCESS;
}

// MDWF_VERBOSE=1: one line per reliable update / residual check on stderr; 2: also the FP64
// residual at every incremental update (diagnostic: costs one FP64 M_pc per update)
static int verbose_level() {
  static const int v = [] { const char* e = getenv("MDWF_VERBOSE"); return e ? atoi(e) : 0; }();
  return v;
}
static bool verbose() { return verbose_level() > 0; }

// CG on M_pc^+ M_pc for the odd-parity system M_pc x = bt (nrhs at once).
// prec == F64: plain FP64 CG; otherwise mixed precision with reliable updates.
int cg_solve(mdwf_ctx* c, const Field& bt, const Field& x64, const mdwf_solve_params* sp, SolveState* S,
             cudaStream_t st) {
  const int nrhs = bt.nrhs;
  const bool mixed = sp->sloppy_prec != F64;
  const int P = sp->sloppy_prec;
  const int form = sp->pc_form;
  CGSet v;
  CKS(make_cgset(c, P, mixed ? F32 : F64, nrhs, form, &v));
  Field res, r64;
  CKS(ws_half(c, "res64", F64, nrhs, &res));
  if (!mixed) CKS(ws_half(c, "r64", F64, nrhs, &r64));   // the plain FP64 CG's normal residual
  CK(cudaMemsetAsync(x64.data, 0, field_bytes_of(x64, F64), st));
  CK(cudaMemsetAsync(v.x.data, 0, field_bytes_of(v.x, v.prec_x), st));
  if (v.x.norm) CK(cudaMemsetAsync(v.x.norm, 0, (size_t)c->vh * nrhs * c->Ls * 4, st));

  const Ops o = ops_of(c, c->prm.mf);
  std::vector<double> tmp;
  CKS(norm2(c, F64, bt, S->bnorm2, st));
  // r = M^+ b~ ; p = r ; phat = D5 p.  The inner (normal-equation) residual only needs
  // the inner precision relative to itself, so the mixed solver forms it in FP32.
  Field r32, res32;
  std::vector<double> g0;
  if (mixed) {
    CKS(ws_half(c, "r32", F32, nrhs, &r32));
    CKS(ws_half(c, "res32", F32, nrhs, &res32));
    CKS(sl_convert(c, F32, res32, F64, bt, false, false, st));
    CKS(apply_Mdag(c, form, F32, res32, r32, st));
    CKS(norm2(c, F32, r32, g0, st));
    CKS(sl_convert(c, P, v.r, F32, r32, false, false, st));
    // FP64 residual of x64 = 0
    CK(cudaMemcpyAsync(res.data, bt.data, field_bytes_of(bt, F64), cudaMemcpyDeviceToDevice, st));
  } else {
    CKS(apply_Mdag(c, form, F64, bt, r64, st));
    CKS(norm2(c, F64, r64, g0, st));
    CK(cudaMemcpyAsync(v.r.data, r64.data, field_bytes_of(r64, F64), cudaMemcpyDeviceToDevice, st));
  }
  CK(cudaMemcpyAsync(v.p.data, v.r.data, field_bytes_of(v.r, P), cudaMemcpyDeviceToDevice, st));
  if (v.r.norm) CK(cudaMemcpyAsync(v.p.norm, v.r.norm, (size_t)c->vh * nrhs * c->Ls * 4, cudaMemcpyDeviceToDevice, st));
  if (form != MDWF_PC_SYM) CKS(sl_chain(c, P, v.ph, v.p, chain(o.D5(false)), 1.0, nullptr, 0.0, o.mf, st));

  for (int r = 0; r < nrhs; r++) {
    if (!std::isfinite(S->bnorm2[r]) || !std::isfinite(g0[r])) {
      g_last_error = "source is not finite (NaN or Inf)";
      return MDWF_ERR_BREAKDOWN;
    }
  }
  S->nrhs = nrhs;
  S->true_rel.assign(nrhs, 1.0);
  S->done.assign(nrhs, 0);
  S->iters.assign(nrhs, 0);
  std::vector<int> since_ru(nrhs, 0);
  for (int r = 0; r < nrhs; r++) {
    CGScalars& s = c->cg_host[r];
    memset(&s, 0, sizeof s);
    s.gamma = g0[r];
    s.maxr2 = g0[r];
    s.stop2 = sp->tol * sp->tol * g0[r];
    s.active = (S->bnorm2[r] > 0.0 && g0[r] > 0.0) ? 1 : 0;
    if (!s.active) { S->done[r] = 1; S->true_rel[r] = 0.0; }
  }
  CKS(push_scalars(c, nrhs, st));

  const int interval = std::max(1, sp->check_interval);
  int ru_since_anchor = 0;
  // |res|^2 at the last FP64 residual (x = 0 at the start: res = b~ exactly)
  std::vector<double> anchor_r2 = S->bnorm2;
  constexpr double kAnchorRatio = 1.6e5;   // 1 % / eps32 (6e-8)
  constexpr int kMaxIncremental = 8;       // at most this many incremental updates in a row
  bool x_fresh = false;   // res holds the FP64 residual of the current x (no iterations since)
  int it = 0;
  bool first = true;
  int status = MDWF_SUCCESS;
  while (true) {
    bool all_done = true;
    for (int r = 0; r < nrhs; r++) all_done &= (bool)S->done[r];
    if (all_done) break;
    if (it >= sp->maxiter) { status = MDWF_ERR_NOT_CONVERGED; break; }
    const int n = std::min(interval, sp->maxiter - it);
    // the first block of iterations runs eagerly so that tuning and allocation finish
    // before any capture
    CKS(run_iterations(c, v, n, sp->use_graph && !first && n == interval, st));
    first = false;
    x_fresh = false;
    it += n;
    CKS(pull_scalars(c, nrhs, st));
    bool need_true = false, need_ru = false;
    for (int r = 0; r < nrhs; r++) {
      if (S->done[r]) continue;
      S->iters[r] = it;
      since_ru[r] += n;
      const CGScalars& s = c->cg_host[r];
      if (s.breakdown || !(s.gamma == s.gamma)) {
        g_last_error = "CG breakdown";
        return MDWF_ERR_BREAKDOWN;
      }
      if (s.hit) need_true = true;
      if (mixed && (s.gamma < sp->delta * sp->delta * s.maxr2 || since_ru[r] >= sp->ru_interval)) need_ru = true;
    }
    if (!need_true && !need_ru) continue;
    std::vector<double> rr2;
    bool anchor = true;
    if (mixed) {
      // Reliable update.  An FP64 anchor recomputes res = b~ - M x64 in FP64; in between,
      // res -= M x_s with M applied in FP32 to the inner accumulator (its rounding error is
      // ~1e-7 |M| |x_s|, x_s being the correction since the last update), then x64 += x_s.
      // The FP32 evaluations of M x_s since the last anchor leave a rounding error of order
      // eps32 |res at the anchor| in res, so an anchor is due once that could exceed 1 % of
      // the current residual (|res_anchor| / |res| > kAnchorRatio), and whenever the
      // incremental residual says the tolerance is reached: convergence is only declared
      // on an FP64 residual.  (Measured: incremental and FP64 residuals agree to four
      // digits up to a ratio of ~1e4.)  When the inner normal residual hits its stopping
      // value, the incremental residual decides whether an FP64 check is due or the inner
      // target is tightened.
      S->ru++;
      anchor = ru_since_anchor >= kMaxIncremental;
      bool folded = false;   // x_s already added to x64 in this update
      if (!anchor) {
        Field q32, q64;
        CKS(ws_half(c, "ru_q32", F32, nrhs, &q32));
        CKS(ws_half(c, "tr_q", F64, nrhs, &q64));
        CKS(apply_M(c, form, F32, v.x, q32, st));
        CKS(sl_convert(c, F64, q64, F32, q32, false, false, st));
        CKS(sl_axpby(c, F64, &res, res, 1.0, &q64, -1.0, red_store(c, nrhs), st));
        CK(cudaMemcpyAsync(c->red_host, c->red_out, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        rr2.assign(c->red_host, c->red_host + nrhs);
        CKS(sl_convert(c, F64, x64, F32, v.x, true, true, st));
        folded = true;
        ru_since_anchor++;
        for (int r = 0; r < nrhs; r++) {
          if (S->done[r]) continue;
          if (rr2[r] <= sp->tol * sp->tol * S->bnorm2[r]) anchor = true;
          if (anchor_r2[r] > kAnchorRatio * kAnchorRatio * rr2[r]) anchor = true;
        }
      }
      if (anchor) {
        if (!folded) CKS(sl_convert(c, F64, x64, F32, v.x, true, true, st));
        // An anchor that may decide convergence (the inner stop or the incremental
        // residual says the tolerance is reached) runs in native FP64; the others in
        // emulated FP64 when the context allows it, and are redone natively should they
        // find the tolerance reached.
        bool may_finish = false;
        for (int r = 0; r < nrhs; r++) {
          if (S->done[r]) continue;
          if (c->cg_host[r].hit || (!rr2.empty() && rr2[r] <= sp->tol * sp->tol * S->bnorm2[r])) may_finish = true;
        }
        const bool emu = c->prm.f64_emulation && c->prm.t_ranks == 1 && !may_finish;
        {
          EmuScope es(c, emu);
          CKS(true_residual(c, form, bt, x64, res, rr2, st));
        }
        S->fp64_res++;
        if (emu) {
          S->emu_res++;
          bool reached = false;
          for (int r = 0; r < nrhs; r++)
            if (!S->done[r] && rr2[r] <= sp->tol * sp->tol * S->bnorm2[r]) reached = true;
          if (reached) {
            CKS(true_residual(c, form, bt, x64, res, rr2, st));
            S->fp64_res++;
          }
        }
        ru_since_anchor = 0;
        x_fresh = true;
        anchor_r2 = rr2;
      }
    } else {
      CKS(true_residual(c, form, bt, v.x, res, rr2, st));
      S->fp64_res++;
      x_fresh = true;
    }
    if (verbose()) {
      std::vector<double> chk;
      if (mixed && !anchor && verbose_level() >= 2) {
        Field rd;
        CKS(ws_half(c, "res_dbg", F64, nrhs, &rd));
        CKS(true_residual(c, form, bt, x64, rd, chk, st));
      }
      for (int r = 0; r < nrhs; r++) {
        if (S->done[r]) continue;
        fprintf(stderr, "[mdwf] it %d rhs %d update %d %s residual %.3e", it, r, S->ru, anchor ? "fp64" : "incr",
                std::sqrt(rr2[r] / S->bnorm2[r]));
        if (!chk.empty()) fprintf(stderr, " (fp64 %.3e)", std::sqrt(chk[r] / S->bnorm2[r]));
        fprintf(stderr, "%s\n", c->cg_host[r].hit ? " (inner stop)" : "");
      }
    }
    for (int r = 0; r < nrhs; r++) {
      if (S->done[r]) continue;
      S->true_rel[r] = std::sqrt(rr2[r] / S->bnorm2[r]);
      CGScalars& s = c->cg_host[r];
      if (anchor && S->true_rel[r] <= sp->tol) {   // convergence only on an FP64 residual
        S->done[r] = 1;
        s.active = 0;
      } else if (s.hit) {
        // the normal residual under-estimated the true one: tighten proportionally
        const double ratio = sp->tol / S->true_rel[r];
        s.stop2 = s.gamma * ratio * ratio * 0.5;
        s.hit = 0;
      }
    }
    bool finished = true;
    for (int r = 0; r < nrhs; r++) finished &= (bool)S->done[r];
    if (finished) break;
    if (mixed) {
      // r = M^+ (b~ - M x) with the FP64 residual rounded to FP32 (relative precision of
      // the inner iteration is all it needs), requantised to the inner storage
      CKS(sl_convert(c, F32, res32, F64, res, false, false, st));
      CKS(apply_Mdag(c, form, F32, res32, r32, st));
      std::vector<double> g, rp;
      CKS(norm2(c, F32, r32, g, st));
      CKS(sl_convert(c, P, v.r, F32, r32, false, false, st));
      // restore <r, p> = |r|^2 for the kept search direction: p += (|r|^2 - <r,p>)/|r|^2 r
      CKS(dot(c, P, v.r, v.p, rp, st));
      std::vector<double> coef(nrhs, 0.0);
      for (int r = 0; r < nrhs; r++) {
        CGScalars& s = c->cg_host[r];
        if (S->done[r]) { s.active = 0; continue; }
        s.gamma = g[r];
        s.maxr2 = g[r];
        s.hit = 0;
        if (s.stop2 > 0.0 && g[r] <= s.stop2) s.stop2 = g[r] * 0.5;
        since_ru[r] = 0;
        coef[r] = g[r] > 0.0 ? (g[r] - rp[r]) / g[r] : 0.0;
      }
      CKS(rhs_axpy(c, P, v.p, v.r, coef, st));
      if (form != MDWF_PC_SYM) CKS(sl_chain(c, P, v.ph, v.p, chain(o.D5(false)), 1.0, nullptr, 0.0, o.mf, st));
    }
    CKS(push_scalars(c, nrhs, st));
  }
  if (!mixed) CK(cudaMemcpyAsync(x64.data, v.x.data, field_bytes_of(x64, F64), cudaMemcpyDeviceToDevice, st));
  for (int r = 0; r < nrhs; r++) S->iters[r] = S->iters[r] ? S->iters[r] : it;
  // final FP64 true residual, unless the last check already computed it for this x
  if (!x_fresh) {
    if (mixed) CKS(sl_convert(c, F64, x64, F32, v.x, true, true, st));
    std::vector<double> rr2;
    CKS(true_residual(c, form, bt, x64, res, rr2, st));
    S->fp64_res++;
    for (int r = 0; r < nrhs; r++) S->true_rel[r] = S->bnorm2[r] > 0 ? std::sqrt(rr2[r] / S->bnorm2[r]) : 0.0;
  }
  return status;
}

// ---------------------------------------------------------------- gamma basis (host, for contractions)
typedef std::complex<double> cd;
struct M4 { cd m[4][4]; };
M4 mzero() { M4 r; for (auto& row : r.m) for (auto& x : row) x = 0; return r; }
M4 mmul(const M4& a, const M4& b) {
  M4 r = mzero();
  for (int i = 0; i < 4; i++) for (int j = 0; j < 4; j++) for (int k = 0; k < 4; k++) r.m[i][j] += a.m[i][k] * b.m[k][j];
  return r;
}
M4 mdag(const M4& a) { M4 r; for (int i = 0; i < 4; i++) for (int j = 0; j < 4; j++) r.m[i][j] = std::conj(a.m[j][i]); return r; }
// chiral basis: gamma_mu = [[0, X], [X^+, 0]], X_k = i sigma_k, X_t = 1
M4 gamma_mu(int mu) {
  const cd I(0, 1);
  cd X[2][2];
  if (mu == 0) { X[0][0] = 0; X[0][1] = I; X[1][0] = I; X[1][1] = 0; }
  else if (mu == 1) { X[0][0] = 0; X[0][1] = 1; X[1][0] = -1.0; X[1][1] = 0; }
  else if (mu == 2) { X[0][0] = I; X[0][1] = 0; X[1][0] = 0; X[1][1] = -I; }
  else { X[0][0] = 1; X[0][1] = 0; X[1][0] = 0; X[1][1] = 1; }
  M4 g = mzero();
  for (int a = 0; a < 2; a++) for (int b = 0; b < 2; b++) { g.m[a][2 + b] = X[a][b]; g.m[2 + b][a] = std::conj(X[a][b]); }
  return g;
}

// In-process exchange among the partitions of one lattice held by contexts of this
// process, each driven by its own host thread: publish the send faces, meet at a host
// barrier, copy the neighbours' faces into the receive buffers on this context's
// stream, meet again so that no partition repacks a face still being read.
struct PartGroup;
struct PartRank {
  PartGroup* group;
  int rank;
};
struct PartGroup {
  int n = 0;
  std::vector<const void*> lo, hi;
  std::vector<PartRank> ranks;
  std::mutex m;
  std::condition_variable cv;
  int waiting = 0;
  long long generation = 0;
  // false when the other partitions did not arrive within the limit
  bool barrier() {
    std::unique_lock<std::mutex> l(m);
    const long long gen = generation;
    if (++waiting == n) {
      waiting = 0;
      generation++;
      cv.notify_all();
      return true;
    }
    if (cv.wait_for(l, std::chrono::seconds(60), [&] { return generation != gen; })) return true;
    waiting--;
    return false;
  }
};

int group_exchange(void* user, const void* send_lo, const void* send_hi, void* recv_lo, void* recv_hi, size_t bytes,
                   void* stream) {
  PartRank* r = (PartRank*)user;
  PartGroup* g = r->group;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(st));   // this partition's faces are packed
  g->lo[r->rank] = send_lo;
  g->hi[r->rank] = send_hi;
  if (!g->barrier()) { g_last_error = "face exchange: the other partitions did not arrive"; return MDWF_ERR_TIMEOUT; }
  CK(cudaMemcpyAsync(recv_hi, g->lo[(r->rank + 1) % g->n], bytes, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(recv_lo, g->hi[(r->rank + g->n - 1) % g->n], bytes, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  if (!g->barrier()) { g_last_error = "face exchange: the other partitions did not arrive"; return MDWF_ERR_TIMEOUT; }
  return MDWF_SUCCESS;
}

}  // namespace

// ======================================================================== C ABI
extern "C" {

void mdwf_default_params(mdwf_params* p) {
  if (!p) return;
  p->dims[0] = p->dims[1] = p->dims[2] = p->dims[3] = 4;
  p->Ls = 8; p->b5 = 1.5; p->c5 = 0.5; p->M5 = 1.3; p->mf = 0.05; p->t_bc = -1.0;
  p->gauge_recon = 18; p->check_su3 = 1;
  p->t_ranks = 1; p->t_rank = 0;
  p->f64_emulation = 1;
}

void mdwf_default_solve_params(mdwf_solve_params* sp) {
  if (!sp) return;
  sp->tol = 1e-10; sp->maxiter = 100000; sp->sloppy_prec = MDWF_PREC_F16; sp->delta = 0.05;
  sp->ru_interval = 100; sp->check_interval = 10; sp->use_graph = 1; sp->location = MDWF_DEVICE;
  sp->full_residual = 0;
  sp->pc_form = MDWF_PC_LEFT;
}

const char* mdwf_strerror(int s) {
  switch (s) {
    case MDWF_SUCCESS: return "success";
    case MDWF_ERR_ARG: return "invalid argument";
    case MDWF_ERR_CUDA: return "CUDA error";
    case MDWF_ERR_OOM: return "out of device memory";
    case MDWF_ERR_NOT_SU3: return "gauge link not in SU(3)";
    case MDWF_ERR_NOT_CONVERGED: return "solver did not converge";
    case MDWF_ERR_BREAKDOWN: return "solver breakdown";
    case MDWF_ERR_TIMEOUT: return "device wait timed out";
    case MDWF_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* mdwf_last_error(void) { return g_last_error.c_str(); }

int mdwf_create(const mdwf_params* p, mdwf_ctx** out) {
  if (!p || !out) { g_last_error = "null pointer"; return MDWF_ERR_ARG; }
  *out = nullptr;
  for (int i = 0; i < 4; i++)
    if (p->dims[i] < 2 || (p->dims[i] & 1)) { g_last_error = "dims must be even and >= 2"; return MDWF_ERR_ARG; }
  if (p->Ls < 2 || p->Ls > MAXLS) { g_last_error = "Ls out of range [2, 32]"; return MDWF_ERR_ARG; }
  if ((double)p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3] >= 4294967296.0) {
    g_last_error = "lattice too large (more than 2^32 sites)"; return MDWF_ERR_ARG;
  }
  if (p->gauge_recon != 18 && p->gauge_recon != 12) { g_last_error = "gauge_recon must be 18 or 12"; return MDWF_ERR_ARG; }
  if (p->gauge_recon == 12 && std::fabs(p->t_bc) != 1.0) { g_last_error = "recon 12 needs t_bc = +-1"; return MDWF_ERR_ARG; }
  if (p->t_ranks < 1 || p->t_rank < 0 || p->t_rank >= p->t_ranks) { g_last_error = "bad t_ranks / t_rank"; return MDWF_ERR_ARG; }
  if (!(p->mf >= 0.0) || !std::isfinite(p->b5) || !std::isfinite(p->c5) || !std::isfinite(p->M5)) {
    g_last_error = "bad Moebius parameters"; return MDWF_ERR_ARG;
  }
  const double al = (4.0 - p->M5) * p->b5 + 1.0;
  if (al == 0.0) { g_last_error = "alpha = (4-M5) b5 + 1 must be nonzero"; return MDWF_ERR_ARG; }
  // the device current now holds every buffer the context will allocate (no device at
  // all is fine here: creation validates and allocates nothing)
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    dev = -1;
    cudaGetLastError();
  }
  mdwf_ctx* c = new mdwf_ctx();
  c->prm = *p;
  c->device = dev;
  c->g.X = p->dims[0]; c->g.Y = p->dims[1]; c->g.Z = p->dims[2]; c->g.T = p->dims[3];
  c->g.Xh = p->dims[0] / 2;
  c->g.fXh = make_fastdiv((uint32_t)c->g.Xh);
  c->g.fY = make_fastdiv((uint32_t)p->dims[1]);
  c->g.fZ = make_fastdiv((uint32_t)p->dims[2]);
  c->vh = (long long)p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3] / 2;
  c->g.vh = c->vh;
  c->slice_vh = (long long)p->dims[0] * p->dims[1] * p->dims[2] / 2;
  c->Ls = p->Ls;
  c->alpha5 = al;
  c->beta5 = (4.0 - p->M5) * p->c5 - 1.0;
  const char* t = getenv("MDWF_TUNE");
  c->tuning = !(t && t[0] == '0');
  const char* tf = getenv("MDWF_TUNE_CACHE");
  if (tf) { c->tune_file = tf; load_tune(c); }
  *out = c;
  return MDWF_SUCCESS;
}

void mdwf_destroy(mdwf_ctx* c) {
  if (!c) return;
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : c->ws) if (kv.second.p) cudaFree(kv.second.p);
  for (int p = 0; p < NPREC; p++)
    for (int q = 0; q < 2; q++) if (c->gauge[p][q]) cudaFree(c->gauge[p][q]);
  if (c->partials) cudaFree(c->partials);
  if (c->counter) cudaFree(c->counter);
  if (c->red_out) cudaFree(c->red_out);
  if (c->cg) cudaFree(c->cg);
  if (c->dev_status) cudaFree(c->dev_status);
  if (c->red_host) cudaFreeHost(c->red_host);
  if (c->cg_host) cudaFreeHost(c->cg_host);
  if (c->status_host) cudaFreeHost(c->status_host);
  delete c;
}

static int ensure_small(mdwf_ctx* c) {
  if (c->red_out) return MDWF_SUCCESS;
  CK(cudaMalloc(&c->red_out, 256 * sizeof(double)));
  CK(cudaMalloc(&c->cg, 64 * sizeof(CGScalars)));
  CK(cudaMemset(c->cg, 0, 64 * sizeof(CGScalars)));
  CK(cudaMalloc(&c->dev_status, sizeof(int)));
  CK(cudaMemset(c->dev_status, 0, sizeof(int)));
  CK(cudaMallocHost(&c->status_host, sizeof(int)));
  CK(cudaMallocHost(&c->red_host, 256 * sizeof(double)));
  CK(cudaMallocHost(&c->cg_host, 64 * sizeof(CGScalars)));
  return MDWF_SUCCESS;
}

int mdwf_load_gauge(mdwf_ctx* c, const double* links, int where, void* stream) {
  if (!c || !links || (where != MDWF_HOST && where != MDWF_DEVICE)) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  CKS(ensure_small(c));
  const long long V = 2 * c->vh;
  const bool ghost = c->prm.t_ranks > 1;   // a leading timeslice from the partition below
  const size_t ubytes = (size_t)(V + (ghost ? 2 * c->slice_vh : 0)) * 4 * 9 * 16;
  const double* dev = links;
  if (where == MDWF_HOST) {
    void* p;
    CKS(ws_get(c, "gauge_user", ubytes, &p));
    CK(cudaMemcpyAsync(p, links, ubytes, cudaMemcpyHostToDevice, st));
    dev = (const double*)p;
  }
  for (int p = 0; p < NPREC; p++)
    for (int q = 0; q < 2; q++)
      if (c->gauge[p][q]) { cudaFree(c->gauge[p][q]); c->gauge[p][q] = nullptr; }
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  const int gs = c->prm.gauge_recon == 12 ? 12 : 18;
  for (int q = 0; q < 2; q++) CK(cudaMalloc(&c->gauge[F64][q], (size_t)c->vh * 8 * gs * sizeof(double)));
  c->gs[F64] = gs;
  void* errp;
  CKS(ws_get(c, "su3err", 64, &errp));
  CK(cudaMemsetAsync(errp, 0, sizeof(double), st));
  GaugeParams gp;
  gp.g = c->g; gp.user = dev; gp.out64[0] = (double*)c->gauge[F64][0]; gp.out64[1] = (double*)c->gauge[F64][1];
  gp.gs = gs; gp.t_bc = c->prm.t_bc; gp.err = (c->prm.check_su3 || gs == 12) ? (double*)errp : nullptr;
  gp.ghost = ghost ? 1 : 0;
  gp.bc_lo = c->prm.t_rank == 0;
  gp.bc_hi = c->prm.t_rank == c->prm.t_ranks - 1;
  CK(launch_gauge_load(gp, st));
  c->launches++;
  double err = 0.0;
  CK(cudaMemcpyAsync(&err, errp, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (gp.err && !(err <= 1e-9)) {
    char b[128];
    snprintf(b, sizeof b, "link not in SU(3): max deviation %.3e", err);
    g_last_error = b;
    c->gauge_loaded = false;
    return MDWF_ERR_NOT_SU3;
  }
  c->gauge_loaded = true;
  return MDWF_SUCCESS;
}

int mdwf_field_bytes(const mdwf_ctx* c, int prec, int nrhs, size_t* bytes) {
  if (prec == PREC_F64E) prec = F64;
  if (!c || !bytes || prec < 0 || prec > 4 || nrhs < 1) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  *bytes = full_bytes(c, prec, nrhs);
  return MDWF_SUCCESS;
}

static int check_nrhs(const mdwf_ctx* c, int nrhs) {
  if (nrhs < 1 || nrhs * c->Ls > MAXTHREADS || nrhs > 64) { g_last_error = "nrhs * Ls must be <= 256"; return MDWF_ERR_ARG; }
  return MDWF_SUCCESS;
}

int mdwf_pack(mdwf_ctx* c, const double* user5d, void* internal, int prec, int nrhs, void* stream) {
  if (prec == PREC_F64E) prec = F64;
  if (!c || !user5d || !internal || prec < 0 || prec > 4 || nrhs < 1) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  PackParams p;
  p.g = c->g; p.Ls = c->Ls; p.nrhs = nrhs; p.user = user5d; p.user_out = nullptr;
  for (int q = 0; q < 2; q++) {
    Field f = view(c, internal, prec, nrhs, q);
    p.data[q] = f.data; p.norm[q] = f.norm;
  }
  CK(launch_pack(prec, p, (cudaStream_t)stream));
  c->launches++;
  c->bytes += (double)2 * c->vh * nrhs * c->Ls * (192.0 + site_bytes(prec));
  return MDWF_SUCCESS;
}

int mdwf_unpack(mdwf_ctx* c, const void* internal, double* user5d, int prec, int nrhs, void* stream) {
  if (prec == PREC_F64E) prec = F64;
  if (!c || !user5d || !internal || prec < 0 || prec > 4 || nrhs < 1) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  PackParams p;
  p.g = c->g; p.Ls = c->Ls; p.nrhs = nrhs; p.user = nullptr; p.user_out = user5d;
  for (int q = 0; q < 2; q++) {
    Field f = view(c, (void*)internal, prec, nrhs, q);
    p.data[q] = f.data; p.norm[q] = f.norm;
  }
  CK(launch_unpack(prec, p, (cudaStream_t)stream));
  c->launches++;
  c->bytes += (double)2 * c->vh * nrhs * c->Ls * (192.0 + site_bytes(prec));
  return MDWF_SUCCESS;
}

int mdwf_apply(mdwf_ctx* c, int op, int prec, const void* in, void* out, int nrhs, void* stream) {
  const bool emu = prec == PREC_F64E;
  if (emu) prec = F64;
  if (!c || !in || !out || prec < 0 || prec > 4 || op < 0 || op >= MDWF_OP_COUNT || in == out) {
    g_last_error = "bad argument"; return MDWF_ERR_ARG;
  }
  if (emu && c->prm.t_ranks > 1) {
    g_last_error = "emulated FP64 is not available on a T-partitioned context";
    return MDWF_ERR_STATE;
  }
  EmuScope scope(c, emu);
  CKS(check_nrhs(c, nrhs));
  if (!c->gauge_loaded) { g_last_error = "no gauge field loaded"; return MDWF_ERR_STATE; }
  CKS(ensure_small(c));
  cudaStream_t st = (cudaStream_t)stream;
  Field fi[2] = {view(c, (void*)in, prec, nrhs, 0), view(c, (void*)in, prec, nrhs, 1)};
  Field fo[2] = {view(c, out, prec, nrhs, 0), view(c, out, prec, nrhs, 1)};
  const Ops o = ops_of(c, c->prm.mf);
  switch (op) {
    case MDWF_OP_HOP_EO: case MDWF_OP_HOP_OE: case MDWF_OP_HOP_EO_DAG: case MDWF_OP_HOP_OE_DAG: {
      const int pout = (op == MDWF_OP_HOP_EO || op == MDWF_OP_HOP_EO_DAG) ? 0 : 1;
      const bool dag = op == MDWF_OP_HOP_EO_DAG || op == MDWF_OP_HOP_OE_DAG;
      Epi e;
      return hop(c, prec, dag, fi[1 - pout], fo[pout], pout, e, red_none(), st);
    }
    case MDWF_OP_HOP_EO_M5INV: case MDWF_OP_HOP_OE_M5INV: {
      const int pout = op == MDWF_OP_HOP_EO_M5INV ? 0 : 1;
      Epi e;
      e.on = true; e.post = chain(o.A5inv(false)); e.mf = o.mf;
      return hop(c, prec, false, fi[1 - pout], fo[pout], pout, e, red_none(), st);
    }
    case MDWF_OP_D5: case MDWF_OP_D5_DAG: case MDWF_OP_M5: case MDWF_OP_M5_DAG: case MDWF_OP_M5INV:
    case MDWF_OP_M5INV_DAG: {
      const bool dag = op == MDWF_OP_D5_DAG || op == MDWF_OP_M5_DAG || op == MDWF_OP_M5INV_DAG;
      SOp so = (op == MDWF_OP_D5 || op == MDWF_OP_D5_DAG) ? o.D5(dag)
               : (op == MDWF_OP_M5 || op == MDWF_OP_M5_DAG) ? o.A5(dag) : o.A5inv(dag);
      for (int q = 0; q < 2; q++) CKS(sl_chain(c, prec, fo[q], fi[q], chain(so), 1.0, nullptr, 0.0, o.mf, st));
      return MDWF_SUCCESS;
    }
    case MDWF_OP_MPC: return apply_mpc(c, prec, fi[1], fo[1], st);
    case MDWF_OP_MPC_DAG: return apply_mpc_dag(c, prec, fi[1], fo[1], st);
    case MDWF_OP_MDAGM: {
      Field t;
      CKS(ws_half(c, "mdagm_t", prec, nrhs, &t));
      CKS(apply_mpc(c, prec, fi[1], t, st));
      return apply_mpc_dag(c, prec, t, fo[1], st);
    }
    case MDWF_OP_MPC_SYM: return apply_mpc_sym(c, prec, fi[1], fo[1], st);
    case MDWF_OP_MPC_SYM_DAG: return apply_mpc_sym_dag(c, prec, fi[1], fo[1], st);
    case MDWF_OP_FULL_D: return apply_full(c, prec, false, fi, fo, c->prm.mf, st);
    case MDWF_OP_FULL_D_DAG: return apply_full(c, prec, true, fi, fo, c->prm.mf, st);
  }
  g_last_error = "unknown op";
  return MDWF_ERR_ARG;
}

int mdwf_solve_multi(mdwf_ctx* c, int nrhs, const double* src, double* sol, const mdwf_solve_params* sp,
                     mdwf_solve_info* info, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!c || !src || !sol || !sp || !info) { g_last_error = "null pointer"; return MDWF_ERR_ARG; }
  CKS(check_nrhs(c, nrhs));
  if (sp->sloppy_prec < 0 || sp->sloppy_prec > 4 || !(sp->tol > 0.0) || sp->maxiter < 1 ||
      (sp->location != MDWF_HOST && sp->location != MDWF_DEVICE) || !(sp->delta > 0.0 && sp->delta < 1.0) ||
      sp->ru_interval < 1 || (sp->pc_form != MDWF_PC_LEFT && sp->pc_form != MDWF_PC_SYM)) {
    g_last_error = "bad solve parameters"; return MDWF_ERR_ARG;
  }
  if (!c->gauge_loaded) { g_last_error = "no gauge field loaded"; return MDWF_ERR_STATE; }
  if (c->prm.t_ranks > 1) {
    g_last_error = "CG on a T-partitioned lattice needs global sums; solve on an undecomposed context";
    return MDWF_ERR_STATE;
  }
  CKS(ensure_small(c));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ubytes = (size_t)nrhs * c->Ls * 2 * c->vh * 12 * 16;
  const double* dsrc = src;
  double* dsol = sol;
  if (sp->location == MDWF_HOST) {
    void *a, *b;
    CKS(ws_get(c, "user_src", ubytes, &a));
    CKS(ws_get(c, "user_sol", ubytes, &b));
    CK(cudaMemcpyAsync(a, src, ubytes, cudaMemcpyHostToDevice, st));
    dsrc = (const double*)a;
    dsol = (double*)b;
  }
  // pack b (FP64 internal), prepare b~_o = A5^-1 (b_o + H_oe D5 A5^-1 b_e / 2)
  void* bint;
  CKS(ws_get(c, "b_int", full_bytes(c, F64, nrhs), &bint));
  CKS(mdwf_pack(c, dsrc, bint, F64, nrhs, st));
  Field b[2] = {view(c, bint, F64, nrhs, 0), view(c, bint, F64, nrhs, 1)};
  const Ops o = ops_of(c, c->prm.mf);
  Field te, bt, xo;
  CKS(ws_half(c, "prep_t", F64, nrhs, &te));
  CKS(ws_half(c, "btilde", F64, nrhs, &bt));
  void* xint;
  CKS(ws_get(c, "x_int", full_bytes(c, F64, nrhs), &xint));
  Field x[2] = {view(c, xint, F64, nrhs, 0), view(c, xint, F64, nrhs, 1)};
  xo = x[1];
  // the FP64 hops of preparing b~ and reconstructing x_e run in emulated FP64 in a mixed
  // solve when the context allows it (their ~1e-14 relative rounding is far below the
  // tolerance, and the convergence check is native FP64)
  const bool emu = sp->sloppy_prec != F64 && c->prm.f64_emulation && c->prm.t_ranks == 1;
  CKS(sl_chain(c, F64, te, b[0], chain(o.A5inv(false), o.D5(false)), 1.0, nullptr, 0.0, o.mf, st));
  {
    EmuScope es(c, emu);
    Epi e;
    e.on = true; e.hc = 0.5; e.center = b[1]; e.fin = chain(o.A5inv(false)); e.mf = o.mf;
    CKS(hop(c, F64, false, te, bt, 1, e, red_none(), st));
  }
  SolveState S;
  const bool sym = sp->pc_form == MDWF_PC_SYM;
  Field rhs = bt;
  if (sym) {   // the symmetric form solves M_sym y = D5 b~_o
    CKS(ws_half(c, "btsym", F64, nrhs, &rhs));
    CKS(sl_chain(c, F64, rhs, bt, chain(o.D5(false)), 1.0, nullptr, 0.0, o.mf, st));
  }
  const int cgs = cg_solve(c, rhs, xo, sp, &S, st);
  if (cgs != MDWF_SUCCESS && cgs != MDWF_ERR_NOT_CONVERGED) return cgs;
  // reconstruct x_e = A5^-1 (b_e + H_eo D5 x_o / 2); te = D5 x_o
  if (sym) {   // xo holds y = D5 x_o: te = y, x_o = D5^-1 y
    CK(cudaMemcpyAsync(te.data, xo.data, field_bytes_of(xo, F64), cudaMemcpyDeviceToDevice, st));
    CKS(sl_chain(c, F64, xo, te, chain(o.D5inv(false)), 1.0, nullptr, 0.0, o.mf, st));
  } else {
    CKS(sl_chain(c, F64, te, xo, chain(o.D5(false)), 1.0, nullptr, 0.0, o.mf, st));
  }
  {
    EmuScope es(c, emu);
    Epi e;
    e.on = true; e.hc = 0.5; e.center = b[0]; e.fin = chain(o.A5inv(false)); e.mf = o.mf;
    CKS(hop(c, F64, false, te, x[0], 0, e, red_none(), st));
  }
  std::vector<double> full_rel(nrhs, -1.0);
  if (sp->full_residual) {
    void* dint;
    CKS(ws_get(c, "d_int", full_bytes(c, F64, nrhs), &dint));
    Field d[2] = {view(c, dint, F64, nrhs, 0), view(c, dint, F64, nrhs, 1)};
    CKS(apply_full(c, F64, false, x, d, c->prm.mf, st));
    std::vector<double> rn(nrhs, 0.0), bn(nrhs, 0.0), t;
    for (int q = 0; q < 2; q++) {
      CKS(sl_axpby(c, F64, &d[q], b[q], 1.0, &d[q], -1.0, red_store(c, nrhs), st));
      CK(cudaMemcpyAsync(c->red_host, c->red_out, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int r = 0; r < nrhs; r++) rn[r] += c->red_host[r];
      CKS(norm2(c, F64, b[q], t, st));
      for (int r = 0; r < nrhs; r++) bn[r] += t[r];
    }
    for (int r = 0; r < nrhs; r++) full_rel[r] = bn[r] > 0 ? std::sqrt(rn[r] / bn[r]) : 0.0;
  }
  CKS(mdwf_unpack(c, xint, dsol, F64, nrhs, st));
  if (sp->location == MDWF_HOST) CK(cudaMemcpyAsync(sol, dsol, ubytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int worst = MDWF_SUCCESS;
  for (int r = 0; r < nrhs; r++) {
    info[r].iterations = S.iters[r];
    info[r].reliable_updates = S.ru;
    info[r].fp64_residuals = S.fp64_res;
    info[r].emulated_residuals = S.emu_res;
    info[r].true_residual = S.true_rel[r];
    info[r].full_residual = full_rel[r];
    info[r].time_ms = ms;
    info[r].status = S.true_rel[r] <= sp->tol ? MDWF_SUCCESS : MDWF_ERR_NOT_CONVERGED;
    if (info[r].status != MDWF_SUCCESS) worst = info[r].status;
  }
  return worst;
}

int mdwf_solve(mdwf_ctx* c, const double* src, double* sol, const mdwf_solve_params* sp, mdwf_solve_info* info,
               void* stream) {
  return mdwf_solve_multi(c, 1, src, sol, sp, info, stream);
}

// ---------------------------------------------------------------- physics helpers
static int stage_in(mdwf_ctx* c, const char* name, const double* p, size_t bytes, int where, cudaStream_t st,
                    const double** dev) {
  if (where == MDWF_DEVICE) { *dev = p; return MDWF_SUCCESS; }
  void* d;
  CKS(ws_get(c, name, bytes, &d));
  CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, st));
  *dev = (const double*)d;
  return MDWF_SUCCESS;
}
static int stage_out(mdwf_ctx* c, const char* name, double* p, size_t bytes, int where, double** dev) {
  if (where == MDWF_DEVICE) { *dev = p; return MDWF_SUCCESS; }
  void* d;
  CKS(ws_get(c, name, bytes, &d));
  *dev = (double*)d;
  return MDWF_SUCCESS;
}
static int finish_out(double* host, const double* dev, size_t bytes, int where, cudaStream_t st) {
  if (where == MDWF_HOST) {
    CK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return MDWF_SUCCESS;
}

int mdwf_make_source_4d(mdwf_ctx* c, const double* src4d, double* src5d, int nrhs, int where, void* stream) {
  if (!c || !src4d || !src5d || (where != MDWF_HOST && where != MDWF_DEVICE)) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  CKS(check_nrhs(c, nrhs));
  if (!c->gauge_loaded) { g_last_error = "no gauge field loaded"; return MDWF_ERR_STATE; }
  CKS(ensure_small(c));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t b4 = (size_t)nrhs * 2 * c->vh * 12 * 16, b5 = b4 * c->Ls;
  const double* in;
  double* out;
  CKS(stage_in(c, "src4_in", src4d, b4, where, st, &in));
  CKS(stage_out(c, "src5_out", src5d, b5, where, &out));
  // the wall source is built in the output buffer, packed, and the result unpacked over it;
  // the packed fields share the solver's FP64 source / solution workspaces (a context runs
  // one call at a time), so injecting costs no memory beyond what a solve of the same nrhs
  // holds anyway
  SrcParams sp;
  sp.g = c->g; sp.Ls = c->Ls; sp.nrhs = nrhs; sp.in = in; sp.out = out;
  CK(launch_embed_wall(sp, st));
  c->launches++;
  void *wi, *di;
  CKS(ws_get(c, "b_int", full_bytes(c, F64, nrhs), &wi));
  CKS(ws_get(c, "x_int", full_bytes(c, F64, nrhs), &di));
  CKS(mdwf_pack(c, out, wi, F64, nrhs, st));
  Field fi[2] = {view(c, wi, F64, nrhs, 0), view(c, wi, F64, nrhs, 1)};
  Field fo[2] = {view(c, di, F64, nrhs, 0), view(c, di, F64, nrhs, 1)};
  {
    EmuScope es(c, c->prm.f64_emulation != 0);   // emulated FP64 where the context allows it
    CKS(apply_full(c, F64, false, fi, fo, 1.0, st));  // Pauli-Villars D(mf = 1)
  }
  CKS(mdwf_unpack(c, di, out, F64, nrhs, st));
  return finish_out(src5d, out, b5, where, st);
}

int mdwf_project_4d(mdwf_ctx* c, const double* sol5d, double* q4d, int nrhs, int where, void* stream) {
  if (!c || !sol5d || !q4d || nrhs < 1 || (where != MDWF_HOST && where != MDWF_DEVICE)) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  CKS(ensure_small(c));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t b4 = (size_t)nrhs * 2 * c->vh * 12 * 16, b5 = b4 * c->Ls;
  const double* in;
  double* out;
  CKS(stage_in(c, "prj_in", sol5d, b5, where, st, &in));
  CKS(stage_out(c, "prj_out", q4d, b4, where, &out));
  SrcParams sp;
  sp.g = c->g; sp.Ls = c->Ls; sp.nrhs = nrhs; sp.in = in; sp.out = out;
  CK(launch_project4d(sp, st));
  c->launches++;
  return finish_out(q4d, out, b4, where, st);
}

// 4D sources -> 4D propagator columns: injection, batched solve and projection chained on
// the device through one 5D workspace (the solve has packed its source before it writes
// its solution, so the two share it); only the 4D fields cross to the host.
int mdwf_propagator(mdwf_ctx* c, int nrhs, const double* src4d, double* q4d, int where,
                    const mdwf_solve_params* sp, mdwf_solve_info* info, void* stream) {
  if (!c || !src4d || !q4d || !sp || !info || (where != MDWF_HOST && where != MDWF_DEVICE)) {
    g_last_error = "bad argument"; return MDWF_ERR_ARG;
  }
  CKS(check_nrhs(c, nrhs));
  if (!c->gauge_loaded) { g_last_error = "no gauge field loaded"; return MDWF_ERR_STATE; }
  CKS(ensure_small(c));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t b4 = (size_t)nrhs * 2 * c->vh * 12 * 16, b5 = b4 * c->Ls;
  const double* in;
  double* out;
  CKS(stage_in(c, "prop_src4", src4d, b4, where, st, &in));
  CKS(stage_out(c, "prop_q4", q4d, b4, where, &out));
  void* f5;
  CKS(ws_get(c, "prop_5d", b5, &f5));
  CKS(mdwf_make_source_4d(c, in, (double*)f5, nrhs, MDWF_DEVICE, stream));
  mdwf_solve_params dsp = *sp;
  dsp.location = MDWF_DEVICE;
  const int rs = mdwf_solve_multi(c, nrhs, (const double*)f5, (double*)f5, &dsp, info, stream);
  if (rs != MDWF_SUCCESS && rs != MDWF_ERR_NOT_CONVERGED) return rs;
  CKS(mdwf_project_4d(c, (const double*)f5, out, nrhs, MDWF_DEVICE, stream));
  CKS(finish_out(q4d, out, b4, where, st));
  return rs;
}

int mdwf_fh_source(mdwf_ctx* c, const double* q4d, double* out4d, int nrhs, int where, void* stream) {
  if (!c || !q4d || !out4d || nrhs < 1 || (where != MDWF_HOST && where != MDWF_DEVICE)) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  CKS(ensure_small(c));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t b4 = (size_t)nrhs * 2 * c->vh * 12 * 16;
  const double* in;
  double* out;
  CKS(stage_in(c, "fh_in", q4d, b4, where, st, &in));
  CKS(stage_out(c, "fh_out", out4d, b4, where, &out));
  SrcParams sp;
  sp.g = c->g; sp.Ls = c->Ls; sp.nrhs = nrhs; sp.in = in; sp.out = out;
  CK(launch_fh_source(sp, st));
  c->launches++;
  return finish_out(out4d, out, b4, where, st);
}

int mdwf_contract_nucleon(mdwf_ctx* c, const double* u1, const double* d, const double* u2, double* corr, int where,
                          void* stream) {
  if (!c || !u1 || !d || !u2 || !corr || (where != MDWF_HOST && where != MDWF_DEVICE)) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  CKS(ensure_small(c));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t pb = (size_t)12 * 2 * c->vh * 12 * 16;
  const double *a, *b, *e;
  CKS(stage_in(c, "nuc_u1", u1, pb, where, st, &a));
  CKS(stage_in(c, "nuc_d", d, pb, where, st, &b));
  CKS(stage_in(c, "nuc_u2", u2, pb, where, st, &e));
  double* out;
  CKS(stage_out(c, "nuc_out", corr, (size_t)c->g.T * 16, where, &out));
  void* site;
  CKS(ws_get(c, "nuc_site", (size_t)2 * c->vh * 16, &site));
  NucMats m;
  nucleon_mats(&m);
  CK(launch_nucleon(c->g, m, a, b, e, (double*)site, out, st));
  c->launches += 2;
  return finish_out(corr, out, (size_t)c->g.T * 16, where, st);
}

int mdwf_fh_effective_coupling(const double* c2, const double* c3, double* geff, int T) {
  if (!c2 || !c3 || !geff || T < 2) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  std::vector<double> R(T);
  for (int t = 0; t < T; t++) {
    const cd C(c2[2 * t], c2[2 * t + 1]), F(c3[2 * t], c3[2 * t + 1]);
    if (!(std::abs(C) > 0.0) || !std::isfinite(std::abs(C))) { g_last_error = "C(t) is zero or not finite"; return MDWF_ERR_ARG; }
    R[t] = (F / C).real();
  }
  for (int t = 0; t + 1 < T; t++) geff[t] = R[t + 1] - R[t];
  return MDWF_SUCCESS;
}

int mdwf_set_tuning(mdwf_ctx* c, int enable) {
  if (!c) return MDWF_ERR_ARG;
  c->tuning = enable != 0;
  return MDWF_SUCCESS;
}

int mdwf_tune_entries(const mdwf_ctx* c, int* count) {
  if (!c || !count) return MDWF_ERR_ARG;
  *count = (int)c->tune.size();
  return MDWF_SUCCESS;
}

int mdwf_tune_entry(const mdwf_ctx* c, int i, char* key, int keylen, int* ns, double* ms) {
  if (!c || i < 0 || i >= (int)c->tune.size()) return MDWF_ERR_ARG;
  auto it = c->tune.begin();
  std::advance(it, i);
  if (key && keylen > 0) {
    strncpy(key, it->first.c_str(), keylen - 1);
    key[keylen - 1] = 0;
  }
  if (ns) *ns = it->second.ns;
  if (ms) *ms = it->second.ms;
  return MDWF_SUCCESS;
}

long long mdwf_launch_count(const mdwf_ctx* c) { return c ? c->launches : 0; }

int mdwf_set_face_exchange(mdwf_ctx* c, mdwf_face_exchange_fn fn, void* user) {
  if (!c) { g_last_error = "null context"; return MDWF_ERR_ARG; }
  c->xfn = fn;
  c->xuser = user;
  return MDWF_SUCCESS;
}

int mdwf_face_bytes(const mdwf_ctx* c, int prec, int nrhs, size_t* bytes) {
  if (!c || !bytes || prec < 0 || prec > 4 || nrhs < 1) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  *bytes = face_bytes_of(c, prec, nrhs);
  return MDWF_SUCCESS;
}

int mdwf_set_face_buffers(mdwf_ctx* c, void* send_lo, void* send_hi, void* recv_lo, void* recv_hi, size_t bytes) {
  if (!c) { g_last_error = "null context"; return MDWF_ERR_ARG; }
  const bool none = !send_lo && !send_hi && !recv_lo && !recv_hi;
  if (!none && (!send_lo || !send_hi || !recv_lo || !recv_hi || bytes == 0)) {
    g_last_error = "face buffers: all four or none";
    return MDWF_ERR_ARG;
  }
  c->user_faces[0] = send_lo; c->user_faces[1] = send_hi;
  c->user_faces[2] = recv_lo; c->user_faces[3] = recv_hi;
  c->user_face_bytes = none ? 0 : bytes;
  return MDWF_SUCCESS;
}

int mdwf_group_partitions(mdwf_ctx* const* ctxs, int n) {
  if (!ctxs || n < 1) { g_last_error = "bad argument"; return MDWF_ERR_ARG; }
  for (int k = 0; k < n; k++) {
    if (!ctxs[k] || ctxs[k]->prm.t_ranks != n || ctxs[k]->prm.t_rank != k) {
      g_last_error = "ctxs[k] must be partition k of n";
      return MDWF_ERR_ARG;
    }
    for (int i = 0; i < 4; i++)
      if (ctxs[k]->prm.dims[i] != ctxs[0]->prm.dims[i] || ctxs[k]->Ls != ctxs[0]->Ls) {
        g_last_error = "partitions of one lattice have the same local shape";
        return MDWF_ERR_ARG;
      }
  }
  auto g = std::make_shared<PartGroup>();
  g->n = n;
  g->lo.assign(n, nullptr);
  g->hi.assign(n, nullptr);
  g->ranks.resize(n);
  for (int k = 0; k < n; k++) {
    g->ranks[k].group = g.get();
    g->ranks[k].rank = k;
    ctxs[k]->group = g;
    ctxs[k]->xfn = group_exchange;
    ctxs[k]->xuser = &g->ranks[k];
  }
  return MDWF_SUCCESS;
}

double mdwf_algorithmic_bytes(const mdwf_ctx* c) { return c ? c->bytes : 0.0; }

}  // extern "C"

// ---------------------------------------------------------------- internal accessors
// (used by translation units that must not touch the context's allocations)
namespace mdwf {

bool ctx_geom(const mdwf_ctx* c, Geom* g) {
  if (!c || !g) return false;
  *g = c->g;
  return true;
}

int ctx_device(const mdwf_ctx* c) { return c ? c->device : -1; }

// Spin matrices of the nucleon contraction in the library's chiral basis.
void nucleon_mats(NucMats* m) {
  const M4 g5 = mmul(mmul(gamma_mu(0), gamma_mu(1)), mmul(gamma_mu(2), gamma_mu(3)));
  const M4 cg5 = mmul(mmul(gamma_mu(1), gamma_mu(3)), g5);
  const M4 cg5b = mmul(mmul(gamma_mu(3), mdag(cg5)), gamma_mu(3));
  const M4 g4 = gamma_mu(3);
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      m->car[i * 4 + j] = cg5.m[i][j].real(); m->cai[i * 4 + j] = cg5.m[i][j].imag();
      m->cbr[i * 4 + j] = cg5b.m[i][j].real(); m->cbi[i * 4 + j] = cg5b.m[i][j].imag();
      const cd pv = 0.5 * ((i == j ? 1.0 : 0.0) + g4.m[i][j]);
      m->pr[i * 4 + j] = pv.real(); m->pi[i * 4 + j] = pv.imag();
    }
}

}  // namespace mdwf
