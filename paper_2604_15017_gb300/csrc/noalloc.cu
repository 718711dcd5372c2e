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
  unsigned char* scratch = nullptr;  // device address of g_envlog_scratch on this device
  int num_sms = 0;
};
DeviceSetup g_setup[MAX_DEVICES];
std::mutex g_setup_lock;

// once per device, with that device current: resolve the array's device address (host code
// cannot use the symbol itself) and the launch shape
int setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lk(g_setup_lock);
  DeviceSetup& s = g_setup[dev];
  if (!s.done) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_envlog_scratch) != cudaSuccess) return US_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return US_ERR_CUDA;
    if (usrt::image_set_attrs(4096) != cudaSuccess) return US_ERR_CUDA;
    s.scratch = (unsigned char*)p;
    s.num_sms = sms;
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
  unsigned long long* key = (unsigned long long*)s->scratch;  // zeroed by the launch below
  float* env = (float*)(s->scratch + NOALLOC_KEY_BYTES);
  usrt::launch_envlog(im, irf_dev, env, key, bmode_dev, s->num_sms * 8, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? US_OK : US_ERR_CUDA;
}
