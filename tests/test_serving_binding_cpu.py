"""Host logic of the serving binding, against a fake library (no GPU): the binding keeps each
request's tensors alive while the server may still touch them, and lets them go once the request
has finished, whether it completed or failed; a timeout keeps them."""
import pytest

import paper_2508_19138_gb300 as pkg
from paper_2508_19138_gb300 import _native as N
from paper_2508_19138_gb300 import serving


class FakeLib:
    def __init__(self, state, rc):
        self.state, self.rc = state, rc

    def _answer(self, state_ref):
        state_ref._obj.value = self.state
        return self.rc

    def bt_server_wait(self, handle, ticket, timeout_s, state_ref):
        return self._answer(state_ref)

    def bt_server_poll(self, handle, ticket, state_ref):
        return self._answer(state_ref)

    def bt_server_destroy(self, handle):
        return N.BT_OK


@pytest.mark.parametrize("call,state,rc,released,raises", [
    ("wait", 2, N.BT_OK, True, False),             # completed
    ("wait", 3, N.BT_ERR_SINGULAR, True, True),    # failed: finished, the error is raised
    ("wait", 1, N.BT_ERR_TIMEOUT, False, True),    # still running when the wait gave up
    ("poll", 2, N.BT_OK, True, False),
    ("poll", 3, N.BT_ERR_SINGULAR, True, True),
    ("poll", 1, N.BT_OK, False, False),            # running
    ("poll", 0, N.BT_OK, False, False),            # queued
])
def test_request_tensors_released_once_finished(monkeypatch, call, state, rc, released, raises):
    fake = FakeLib(state, rc)
    monkeypatch.setattr(N, "load", lambda: fake)
    srv = serving.Server(handle=1)
    srv.keep[7] = ("tensors",)
    fn = serving.bt_server_wait if call == "wait" else serving.bt_server_poll
    if raises:
        with pytest.raises(pkg.BTError):
            fn(srv, 7)
    else:
        assert fn(srv, 7) == state
    assert (7 not in srv.keep) == released
    srv.close()
