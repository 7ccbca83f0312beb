// Internal hooks between the handle code and the request server (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include "../../include/me.h"

// Enqueue, on the handle's stream, a copy of the last call's rescue count to `dst`
// (host-pinned); returns ME_OK or an error code.
int me_internal_rescued_async(me_handle* h, int* dst);
// Launches of one batch whose size is read on the device (*d_n <= cap; momenta with
// stride cap, weights optional): the main kernel, the float64 rescue of the flagged
// points (mixed precision, subtracted real) and the reduction, on the handle's stream.
// Allocates nothing and never synchronises, so the sequence can be captured in a CUDA
// graph and replayed for any batch size up to cap.  me_internal_prepare_counted (outside
// any capture, after one ordinary call of the kind) sizes the handle's scratch for cap.
int me_internal_prepare_counted(me_handle* h, int me_kind, int64_t cap);
int me_internal_launch_counted(me_handle* h, int me_kind, const double* d_p, const double* d_w, int64_t cap,
                               const int* d_n, double* d_out);
// Final-state masses of the handle's process (outgoing legs in order; at most 4), their
// number, and the handle's stream.
int me_internal_final_masses(me_handle* h, double* masses, int* n_out, cudaStream_t* stream);
// Process id (index into the library's process table) of a name, or -1.
int me_internal_process_id(const char* name);
// Process id of a handle, or -1 for NULL.
int me_internal_handle_process(const me_handle* h);
// Record the thread-local message returned by me_last_error(); returns `code`.
int me_internal_fail(int code, const char* msg);

namespace me {
struct ColourTables;
struct KParams;
}  // namespace me
// Fill host colour tables (the same construction as the per-device set-up).
int me_internal_build_tables(me::ColourTables* tab);
// Validate parameters and fill kernel parameters for a process (tables pointer unset).
int me_internal_kparams(const char* process, const me_params* params, me::KParams* kp, int* pid);
// The same with the device-resident tables of params->device set up and filled in.
int me_internal_device_kparams(const char* process, const me_params* params, me::KParams* kp, int* pid);
// Whether a buffer of CUDA memory type `mem_type` on device `mem_device` can be handed to
// a kernel on `want_device` without peer access (1) or not (0); exported with C linkage.
extern "C" int me_internal_buffer_usable(int mem_type, int mem_device, int want_device);
