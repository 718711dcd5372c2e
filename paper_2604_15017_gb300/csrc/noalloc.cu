// Allocation-free variant of the fused envelope + log-compression stage.
//
// Some callers cannot allocate device memory when they call us: code that runs inside another
// framework's memory pool or under a hard device-memory cap, code that issues work while a
// stream is being captured, and latency-critical serving loops where a first-call allocation
// (and the stream synchronisation a growing workspace needs) is not acceptable.  This entry
// point keeps its scratch (the envelope image and the packed maximum) in a fixed file-scope
// device array instead, and calls no allocator at all.
#include <mutex>

#include "../../include/usrt.h"
#include "image.cuh"

namespace {

// scratch: [0, 256) bytes hold the packed (E_max, argmax) key, then the envelope image
constexpr size_t NOALLOC_KEY_BYTES = 256;
constexpr size_t NOALLOC_BYTES = NOALLOC_KEY_BYTES + sizeof(float) * (size_t)US_ENVLOG_NOALLOC_MAX_PIXELS;
static __device__ __align__(256) unsigned char g_envlog_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
struct DeviceSetup {
  bool done = false;
  unsigned long long ctx_id = 0;     // the CUDA context the set-up was made in
  unsigned char* scratch = nullptr;  // device address of g_envlog_scratch in that context
  int num_sms = 0;
};
DeviceSetup g_setup[MAX_DEVICES];
std::mutex g_setup_lock;

// The current context's unique id, through driver entry points the runtime hands out (the
// library does not link the driver library itself).  A device reset, or a new primary context,
// reloads the module: the array then has a new address and the kernels' shared-memory limits
// are unset, so the set-up is redone whenever the id changes.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
int current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult r1, r2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &r1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &r2) != cudaSuccess ||
        r1 != cudaDriverEntryPointSuccess || r2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return US_ERR_CUDA;
    get_current = (CtxGetCurrentFn)f1;
    get_id = (CtxGetIdFn)f2;
  }
  void* c = nullptr;
  if (get_current(&c) != 0 || !c || get_id(c, id) != 0) return US_ERR_CUDA;
  return US_OK;
}

// once per device and context, with that device current: resolve the array's device address
// (host code cannot use the symbol itself), the kernels' shared-memory limits and the launch
// shape
int setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lk(g_setup_lock);
  DeviceSetup& s = g_setup[dev];
  unsigned long long id = 0;
  if (current_context_id(&id) != US_OK) return US_ERR_CUDA;
  if (!s.done || s.ctx_id != id) {
    s.done = false;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_envlog_scratch) != cudaSuccess) return US_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return US_ERR_CUDA;
    if (usrt::image_set_attrs(4096) != cudaSuccess) return US_ERR_CUDA;
    s.scratch = (unsigned char*)p;
    s.num_sms = sms;
    s.ctx_id = id;
    s.done = true;
  }
  *out = &s;
  return US_OK;
}

}  // namespace

extern "C" int us_envlog_noalloc(const us_img_desc* img, const float* irf_dev, float* bmode_dev, void* stream) {
  if (!img || !irf_dev || !bmode_dev) return US_ERR_ARG;
  if (img->n_lines < 1 || img->n_depth < 16 || img->n_depth > 4096 || (img->n_depth & (img->n_depth - 1)))
    return US_ERR_ARG;
  if ((long long)img->n_lines * img->n_depth > (long long)US_ENVLOG_NOALLOC_MAX_PIXELS) return US_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return US_ERR_CUDA;
  DeviceSetup* s = nullptr;
  const int rc = setup_device(dev, &s);
  if (rc != US_OK) return rc;
  usrt::Img im;
  im.nl = img->n_lines;
  im.nd = img->n_depth;
  im.x0 = img->x0;
  im.x1 = img->x1;
  im.z0 = img->z0;
  im.z1 = img->z1;
  im.dr = img->dr_db;
  im.l1 = img->lambda1;
  im.l2 = img->lambda2;
  im.fnum = img->f_number;
  unsigned long long* key = (unsigned long long*)s->scratch;  // zeroed by the launch below
  float* env = (float*)(s->scratch + NOALLOC_KEY_BYTES);
  // the launches' own status: an error left pending by unrelated earlier work is neither
  // reported nor cleared here
  cudaError_t err = cudaSuccess;
  usrt::launch_envlog(im, irf_dev, env, key, bmode_dev, s->num_sms * 8, (cudaStream_t)stream, nullptr, 0, &err);
  return err == cudaSuccess ? US_OK : US_ERR_CUDA;
}
