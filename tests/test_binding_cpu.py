"""The Python binding's completion-callback trampoline, on the host alone: the
library calls one C function pointer with the token it was given as arg; the
trampoline must run the matching Python callable once, with (ticket, status),
forget it afterwards, and keep an exception raised by the callable out of the
library's thread."""
import ctypes

import paper_1305_3345_gb300 as kg


def test_trampoline_runs_each_callable_once():
    calls = []
    token = next(kg._done_tokens)
    kg._done_callables[token] = lambda t, s: calls.append((t, s))
    kg._done_c(ctypes.c_void_p(token), 2**64 - 1, -2)   # through the C function pointer
    kg._done_c(ctypes.c_void_p(token), 7, 0)            # a second call for the token is ignored
    assert calls == [(2**64 - 1, -2)]
    assert token not in kg._done_callables


def test_trampoline_contains_exceptions(capsys):
    token = next(kg._done_tokens)

    def boom(t, s):
        raise RuntimeError("callback failed")

    kg._done_callables[token] = boom
    kg._done_c(ctypes.c_void_p(token), 1, 0)            # must not raise
    assert "callback failed" in capsys.readouterr().err
    assert token not in kg._done_callables


def test_callback_signature_matches_the_header():
    # void (*kgpu_done_fn)(void *arg, kgpu_ticket ticket, int status)
    assert kg.DONE_FN._restype_ is None
    assert kg.DONE_FN._argtypes_ == (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int)
