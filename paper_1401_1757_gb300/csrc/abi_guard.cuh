// abi_guard.cuh -- no C++ exception crosses the C ABI.  Every exported entry
// point is a function-try-block whose handler maps the exception being
// handled to a status code: std::bad_alloc (a host allocation) to
// RSV_E_NOMEM, anything else (a thread that could not start, ...) to
// RSV_E_ARG, with the message kept on the context when there is one.
#pragma once

#include <exception>
#include <new>

#include "rsv.h"

struct rsv_ctx;

namespace rsv {

// Record msg as the context's last error (when c is not null); returns st.
rsv_status fail_msg(rsv_ctx* c, rsv_status st, const char* msg) noexcept;

// The status of the exception being handled: call only inside a handler.
inline rsv_status host_error(rsv_ctx* c) noexcept {
    try {
        throw;
    } catch (const std::bad_alloc&) {
        return fail_msg(c, RSV_E_NOMEM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail_msg(c, RSV_E_ARG, e.what());
    } catch (...) {
        return fail_msg(c, RSV_E_ARG, "unexpected host error");
    }
}

}  // namespace rsv
