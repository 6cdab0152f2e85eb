// Batched reduced steps: many independent instances (own N, n, p, grid, dt)
// advanced together, one CUDA graph launch per phase of a step.
//
// Each instance keeps its own context (workspace), state and fixed-point
// flags.  At creation the three phases of one step (vp_api.cu: pre = field,
// energies, basis stage and fixed-point set-up, followed by R1 fixed-point
// rounds; rounds = R2 more rounds; post = Z update, tangent velocity, Cayley
// retraction, re-orthonormalisation) are captured for all instances into
// three graphs whose instances are parallel branches.  A step launches the
// first graph, reads the instances' done flags with one small kernel and one
// synchronisation, launches the rounds graph until every instance has
// converged (converged instances return at once from every round kernel), and
// launches the post graph.  The kernels and their order per instance are
// those of vp_basis_update with a warm-started fixed point, so each instance
// gets the same bits as its own vp_basis_update call.
#include "vp_internal.cuh"

#include <algorithm>
#include <cstdarg>
#include <string>
#include <vector>

namespace {

__global__ void k_batch_check(int B, int* const* flags, int* out) {
  __shared__ int pending, maxit;
  if (threadIdx.x == 0) {
    pending = 0;
    maxit = 0;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int* f = flags[b];
    if (!f[0]) atomicAdd(&pending, 1);
    atomicMax(&maxit, f[1]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = pending;
    out[1] = maxit;
  }
}

// After a step: trace rows (p x 2) and iteration counts of every instance into
// the caller's buffers at row `step`.
__global__ void k_batch_gather(int B, const int* __restrict__ p, double* const* src,
                               double* const* dst, int* const* flags, int32_t* const* iters,
                               int64_t step) {
  const int b = blockIdx.x;
  if (b >= B) return;
  const int m = 2 * p[b];
  if (dst[b] && src[b])
    for (int e = threadIdx.x; e < m; e += blockDim.x) dst[b][step * m + e] = src[b][e];
  if (threadIdx.x == 0 && iters[b]) iters[b][step] = flags[b][1];
}

__global__ void k_batch_status(int B, int* const* status, int* out) {
  if (threadIdx.x != 0) return;
  out[0] = 0;
  out[1] = -1;
  for (int b = 0; b < B; ++b)
    if (*status[b] != 0) {
      out[0] = *status[b];
      out[1] = b;
      return;
    }
}

}  // namespace

struct vp_batch {
  int device = 0;
  int B = 0;
  int R1 = 8, R2 = 2;
  vp_step_opts o{};
  std::vector<vp_batch_item> items;
  std::vector<vp_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<InstanceStep*> steps;
  std::vector<double*> trace_tmp;  // p x 2 per instance (device)
  std::vector<double*> kown;       // internal warm-start states (device)
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  size_t nodes[3] = {0, 0, 0};
  // device tables
  int* d_p = nullptr;
  double** d_src = nullptr;
  double** d_dst = nullptr;
  int** d_flags = nullptr;
  int32_t** d_iters = nullptr;
  int** d_status = nullptr;
  int* d_out = nullptr;
  int* h_out = nullptr;  // pinned
  int64_t steps_done = 0;
  int64_t launches = 0;
  std::string err;
};

// Message of the last failed vp_batch_create on this thread.
static thread_local std::string g_create_err;

static vp_status bfail(vp_batch* b, vp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  return s;
}

static void batch_free(vp_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  for (auto& e : b->exec)
    if (e) cudaGraphExecDestroy(e);
  for (auto* s : b->steps) step_free(s);
  for (auto* t : b->trace_tmp)
    if (t) cudaFree(t);
  for (auto* k : b->kown)
    if (k) cudaFree(k);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->joins)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  for (auto* c : b->ctx)
    if (c) vp_ctx_destroy(c);
  for (void* ptr : {(void*)b->d_p, (void*)b->d_src, (void*)b->d_dst, (void*)b->d_flags,
                    (void*)b->d_iters, (void*)b->d_status, (void*)b->d_out})
    if (ptr) cudaFree(ptr);
  if (b->h_out) cudaFreeHost(b->h_out);
  delete b;
}

// Capture phase `ph` (0 pre + R1 rounds, 1 R2 rounds, 2 post) of all instances.
static vp_status capture(vp_batch* b, int ph) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return bfail(b, VP_ECUDA, "stream capture could not start");
  vp_status s = VP_OK;
  cudaEventRecord(b->fork, b->origin);
  for (int i = 0; i < b->B && s == VP_OK; ++i) {
    cudaStreamWaitEvent(b->streams[i], b->fork, 0);
    if (ph == 0) {
      s = step_pre(b->steps[i], b->trace_tmp[i]);
      if (s == VP_OK) s = step_rounds(b->steps[i], b->R1);
    } else if (ph == 1) {
      s = step_rounds(b->steps[i], b->R2);
    } else {
      s = step_post(b->steps[i]);
    }
    if (s != VP_OK) b->err = std::string("instance ") + std::to_string(i) + ": " + vp_last_error(b->ctx[i]);
    cudaEventRecord(b->joins[i], b->streams[i]);
    cudaStreamWaitEvent(b->origin, b->joins[i], 0);
  }
  cudaError_t e = cudaStreamEndCapture(b->origin, &g);
  if (s != VP_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess || !g) return bfail(b, VP_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
  // kernel nodes (the launches a replay makes)
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
  size_t nk = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
  }
  b->nodes[ph] = nk;
  e = cudaGraphInstantiate(&b->exec[ph], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, VP_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  return VP_OK;
}

extern "C" {

vp_status vp_batch_create(vp_batch** out, int device, const vp_batch_item* items, int32_t count,
                          const vp_step_opts* opts, int32_t rounds_first, int32_t rounds_more,
                          size_t scratch_per_instance) {
  if (!out || !items || count < 1 || count > 4096 || !opts || opts->arith < 1 || opts->arith > 2 ||
      rounds_first < 1 || rounds_more < 1 || opts->maxit < 1)
    return VP_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return VP_ECUDA;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  vp_batch* b = new vp_batch();
  b->device = device;
  b->B = count;
  b->R1 = rounds_first;
  b->R2 = rounds_more;
  b->o = *opts;
  b->items.assign(items, items + count);
  vp_status s = VP_OK;
  // on failure the partial batch is freed (its message with it)
  auto done = [&](vp_status code) {
    cudaSetDevice(prev);
    if (code != VP_OK) {
      g_create_err = b->err.empty() ? vp_status_string(code) : b->err;
      batch_free(b);
      *out = nullptr;
      return code;
    }
    *out = b;
    return VP_OK;
  };
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return done(VP_ECUDA);
  b->ctx.assign(count, nullptr);
  b->streams.assign(count, nullptr);
  b->steps.assign(count, nullptr);
  b->trace_tmp.assign(count, nullptr);
  b->kown.assign(count, nullptr);
  b->joins.assign(count, nullptr);
  std::vector<int> hp(count);
  std::vector<double*> hsrc(count), hdst(count);
  std::vector<int*> hflags(count), hstatus(count);
  std::vector<int32_t*> hiters(count);
  for (int i = 0; i < count && s == VP_OK; ++i) {
    const vp_batch_item& it = items[i];
    if (!it.Q_dev || !it.Z_dev || it.p < 1 || it.n < 1 || (it.trace_dev && it.trace_capacity < 1)) {
      s = VP_EINVAL;
      break;
    }
    if (vp_ctx_create(&b->ctx[i], device, scratch_per_instance) != VP_OK) {
      s = bfail(b, VP_ENOMEM, "context of instance %d", i);
      break;
    }
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming) != cudaSuccess) {
      s = VP_ECUDA;
      break;
    }
    double* ks = it.kstate_dev;
    const size_t zb = sizeof(double) * 2 * (size_t)it.n * it.p;
    if (!ks) {
      if (cudaMalloc(&b->kown[i], zb) != cudaSuccess) {
        s = VP_ENOMEM;
        break;
      }
      cudaMemset(b->kown[i], 0, zb);
      ks = b->kown[i];
    }
    if (it.trace_dev && cudaMalloc(&b->trace_tmp[i], sizeof(double) * 2 * it.p) != cudaSuccess) {
      s = VP_ENOMEM;
      break;
    }
    s = step_setup(b->ctx[i], &it.grid, it.N, it.n, it.p, it.Q_dev, it.Z_dev, it.dt, &b->o, ks,
                   b->streams[i], &b->steps[i]);
    if (s != VP_OK) {
      bfail(b, s, "instance %d: %s", i, vp_last_error(b->ctx[i]));
      break;
    }
    hp[i] = it.p;
    hsrc[i] = b->trace_tmp[i];
    hdst[i] = it.trace_dev;
    hflags[i] = step_flags(b->steps[i]);
    hiters[i] = it.iters_dev;
    hstatus[i] = b->ctx[i]->d_status;
  }
  if (s != VP_OK) return done(s);
  const size_t B = count;
  bool ok = cudaMalloc(&b->d_p, sizeof(int) * B) == cudaSuccess &&
            cudaMalloc(&b->d_src, sizeof(double*) * B) == cudaSuccess &&
            cudaMalloc(&b->d_dst, sizeof(double*) * B) == cudaSuccess &&
            cudaMalloc(&b->d_flags, sizeof(int*) * B) == cudaSuccess &&
            cudaMalloc(&b->d_iters, sizeof(int32_t*) * B) == cudaSuccess &&
            cudaMalloc(&b->d_status, sizeof(int*) * B) == cudaSuccess &&
            cudaMalloc(&b->d_out, sizeof(int) * 4) == cudaSuccess &&
            cudaMallocHost(&b->h_out, sizeof(int) * 4) == cudaSuccess;
  if (!ok) return done(VP_ENOMEM);
  cudaMemcpy(b->d_p, hp.data(), sizeof(int) * B, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_src, hsrc.data(), sizeof(double*) * B, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_dst, hdst.data(), sizeof(double*) * B, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_flags, hflags.data(), sizeof(int*) * B, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_iters, hiters.data(), sizeof(int32_t*) * B, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_status, hstatus.data(), sizeof(int*) * B, cudaMemcpyHostToDevice);
  // workspaces are set up and zeroed on the instance streams before capture
  for (auto st : b->streams) cudaStreamSynchronize(st);
  for (int ph = 0; ph < 3 && s == VP_OK; ++ph) s = capture(b, ph);
  if (s == VP_OK && cudaDeviceSynchronize() != cudaSuccess) s = VP_ECUDA;
  return done(s);
}

vp_status vp_batch_step(vp_batch* b, int32_t nsteps, void* stream) {
  if (!b || nsteps < 0) return VP_EINVAL;
  cudaSetDevice(b->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (const auto& it : b->items)
    if (it.trace_dev && b->steps_done + nsteps > it.trace_capacity)
      return bfail(b, VP_EINVAL, "trace capacity %d reached", it.trace_capacity);
  for (int step = 0; step < nsteps; ++step) {
    if (cudaGraphLaunch(b->exec[0], st) != cudaSuccess) return bfail(b, VP_ECUDA, "graph launch");
    b->launches += (int64_t)b->nodes[0];
    int total = b->R1;
    for (;;) {
      k_batch_check<<<1, 256, 0, st>>>(b->B, b->d_flags, b->d_out);
      ++b->launches;
      cudaMemcpyAsync(b->h_out, b->d_out, sizeof(int) * 2, cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) return bfail(b, VP_ECUDA, "step synchronisation");
      if (b->h_out[0] == 0) break;
      // coeff_update marks every instance done by maxit iterations, so this
      // loop ends; the bound below only guards against a broken invariant
      if (total > b->o.maxit + b->R2) return bfail(b, VP_ENOCONV, "fixed point did not finish");
      if (cudaGraphLaunch(b->exec[1], st) != cudaSuccess) return bfail(b, VP_ECUDA, "graph launch");
      b->launches += (int64_t)b->nodes[1];
      total += b->R2;
    }
    if (cudaGraphLaunch(b->exec[2], st) != cudaSuccess) return bfail(b, VP_ECUDA, "graph launch");
    b->launches += (int64_t)b->nodes[2];
    k_batch_gather<<<b->B, 64, 0, st>>>(b->B, b->d_p, b->d_src, b->d_dst, b->d_flags, b->d_iters,
                                         b->steps_done);
    ++b->launches;
    ++b->steps_done;
  }
  k_batch_status<<<1, 32, 0, st>>>(b->B, b->d_status, b->d_out);
  ++b->launches;
  cudaMemcpyAsync(b->h_out, b->d_out, sizeof(int) * 2, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return bfail(b, VP_ECUDA, "step synchronisation");
  if (b->h_out[0] != 0)
    return bfail(b, (vp_status)b->h_out[0], "instance %d reported %s", b->h_out[1],
                 vp_status_string((vp_status)b->h_out[0]));
  return VP_OK;
}

vp_status vp_batch_info(const vp_batch* b, int64_t* steps_done, int64_t* launches,
                        int64_t* graph_nodes) {
  if (!b) return VP_EINVAL;
  if (steps_done) *steps_done = b->steps_done;
  if (launches) *launches = b->launches;
  if (graph_nodes) {
    graph_nodes[0] = (int64_t)b->nodes[0];
    graph_nodes[1] = (int64_t)b->nodes[1];
    graph_nodes[2] = (int64_t)b->nodes[2];
  }
  return VP_OK;
}

const char* vp_batch_last_error(const vp_batch* b) { return b ? b->err.c_str() : g_create_err.c_str(); }

vp_status vp_batch_destroy(vp_batch* b) {
  if (!b) return VP_EINVAL;
  batch_free(b);
  return VP_OK;
}

}  // extern "C"
