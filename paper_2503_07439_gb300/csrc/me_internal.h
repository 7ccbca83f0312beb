// Internal hooks between the handle code and the request server (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include "../../include/me.h"

// Enqueue, on the handle's stream, a copy of the last call's rescue count to `dst`
// (host-pinned); returns ME_OK or an error code.
int me_internal_rescued_async(me_handle* h, int* dst);
// Process id (index into the library's process table) of a name, or -1.
int me_internal_process_id(const char* name);
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
