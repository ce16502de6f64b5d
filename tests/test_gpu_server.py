"""The render server (continuous batching): every result is the same alone and
in the mix; memory and residency limits, malformed requests, bounded waits and
cancellation behave as documented.  Failures are made on the host (budgets,
bad arguments, queued work), never by faulting the GPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    build.build()
    vols = [ph.gaussian_blobs(32, 11), ph.ct_phantom(48, 12),
            ph.gaussian_blobs(40, 13)[:28, :36, :40].copy()]
    tfs = [(ph.tf_random_pl(256, 11), 0.0, 255.0), (ph.tf_ct(512, 12), 0.0, 4095.0),
           (ph.tf_random_pl(64, 13), 0.0, 255.0)]
    return torch, ph, vi, vols, tfs


def make_requests(ph, vi, count, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(count):
        v = int(rng.integers(3))
        W, H = [(32, 24), (48, 40), (64, 64), (57, 31)][int(rng.integers(4))]
        reqs.append(dict(
            vol=v, light=ph.random_direction(rng),
            cam=ph.orbit_camera(ph.random_direction(rng), bool(rng.integers(2)), 2.4),
            n=int([8, 16, 33][rng.integers(3)]), R=int([16, 24, 45][rng.integers(3)]),
            mode=int(rng.integers(1, 4)), fmt=int([vi.F32, vi.F16, vi.UNORM16][rng.integers(3)]),
            W=W, H=H, ert=float([2.0, 0.95][rng.integers(2)])))
    return reqs


def run(env, reqs, slots, together, budget=0, max_resident=0, batching=False):
    torch, ph, vi, vols, tfs = env
    with vi.Server(0, slots=slots, memory_budget=budget, max_resident_volumes=max_resident,
                   batching=batching) as s:
        vids = [s.add_volume(v) for v in vols]
        outs, tickets = [], []
        for q in reqs:
            out = torch.full((q["H"], q["W"], 4), float("nan"), device="cuda")
            tf, vmin, vmax = tfs[q["vol"]]
            t = s.submit(vids[q["vol"]], tf, vmin, vmax, q["light"], q["n"], q["R"], q["mode"],
                         q["cam"], q["W"], q["H"], 0.5, out, format=q["fmt"], ert=q["ert"])
            outs.append(out)
            tickets.append(t)
            if not together:
                assert s.wait(t) == (vi.REQ_DONE, vi.OK)
        for t in tickets:
            assert s.wait(t) == (vi.REQ_DONE, vi.OK)
        stats = s.stats()
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], stats


def test_results_are_identical_alone_and_in_the_mix(env):
    torch, ph, vi, vols, tfs = env
    reqs = make_requests(ph, vi, 16)
    alone, _ = run(env, reqs, slots=1, together=False)
    mixed, stats = run(env, reqs, slots=4, together=True)
    for a, b in zip(alone, mixed):
        assert np.isfinite(a).all()
        assert np.array_equal(a, b)
    assert stats["completed"] == 16 and stats["failed"] == 0


def test_server_frame_equals_context_frame(env):
    """A served frame is the frame a plain context renders from the same inputs."""
    torch, ph, vi, vols, tfs = env
    q = make_requests(ph, vi, 1, seed=5)[0]
    (served,), _ = run(env, [q], slots=2, together=True)
    tf, vmin, vmax = tfs[q["vol"]]
    with vi.Context(0) as c:
        c.load_volume(vols[q["vol"]])
        c.set_transfer_function(tf, vmin, vmax)
        c.set_light(q["light"])
        c.build_attenuation(q["n"], q["R"], q["mode"], format=q["fmt"])
        ref = c.render(q["cam"], q["W"], q["H"], 0.5, ert=q["ert"]).cpu().numpy()
    assert np.array_equal(served, ref)


def test_batched_marches_give_the_same_frames(env):
    """With batching on, the marches of the requests admitted together run as
    batches of persistent launches whose frames wait on the device for their
    slots' stacks: every frame equals the one-slot frame, and the BF16 /
    UNORM16 requests (outside the batches' restrictions) keep their own march."""
    torch, ph, vi, vols, tfs = env
    reqs = make_requests(ph, vi, 24, seed=17)
    for k, q in enumerate(reqs):
        q["fmt"] = [vi.F32, vi.F16, vi.F32, vi.UNORM16][k % 4]
    alone, _ = run(env, reqs, slots=1, together=False)
    for together in (False, True):
        got, stats = run(env, reqs, slots=4, together=together, batching=True)
        for a, b in zip(alone, got):
            assert np.isfinite(a).all()
            assert np.array_equal(a, b)
        assert stats["completed"] == 24 and stats["failed"] == 0
        assert stats["batched_frames"] == sum(q["fmt"] != vi.UNORM16 for q in reqs)
        # How many frames share a batch depends on how fast requests arrive
        # against the scheduler's passes; every batch holds at least one.
        assert 1 <= stats["batches"] <= stats["batched_frames"]


@pytest.mark.parametrize("path", ["graphs", "batching"])
def test_served_frames_match_the_oracle(env, path):
    """Every served frame matches the FP64 oracle, not only the server's own
    one-slot frames: 4 slots, all requests submitted at once, graphs on, mixed
    volumes (uint8 blobs, uint16 ellipsoids, a non-cubic one), TFs, shadow /
    shell / cone and the four storage formats.  Tolerance: the image tolerance
    plus half an ulp of the stack's format; sample counts exact (inside an
    early-termination window, one of its outcomes)."""
    import oracle
    from gpu_common import FORMAT_HALF_ULP, IMAGE_TOL, check_frame, oracle_frame
    torch, ph, vi, vols, tfs = env
    oracle.build()
    reqs = make_requests(ph, vi, 12, seed=21)
    fmts = [vi.F32, vi.F16, vi.BF16, vi.UNORM16]
    for k, q in enumerate(reqs):
        q["fmt"] = fmts[k % 4]
        q["vol"] = k % 3
        q["mode"] = 1 + (k // 4) % 3
    outs, counts = [], []
    with vi.Server(0, slots=4, graphs=path == "graphs", batching=path == "batching") as s:
        vids = [s.add_volume(v) for v in vols]
        tickets = []
        for q in reqs:
            out = torch.full((q["H"], q["W"], 4), float("nan"), device="cuda")
            cnt = torch.full((q["H"], q["W"]), -1, dtype=torch.int32, device="cuda")
            tf, vmin, vmax = tfs[q["vol"]]
            tickets.append(s.submit(vids[q["vol"]], tf, vmin, vmax, q["light"], q["n"], q["R"],
                                    q["mode"], q["cam"], q["W"], q["H"], 0.5, out,
                                    format=q["fmt"], ert=q["ert"], sample_counts=cnt))
            outs.append(out)
            counts.append(cnt)
        for t in tickets:
            assert s.wait(t) == (vi.REQ_DONE, vi.OK)
        st = s.stats()
        if path == "graphs":
            assert st["graph_launches"] == len(reqs)
        else:
            assert st["batched_frames"] == sum(q["fmt"] in (vi.F32, vi.F16) for q in reqs)
    torch.cuda.synchronize()
    for q, out, cnt in zip(reqs, outs, counts):
        tf, vmin, vmax = tfs[q["vol"]]
        sc = ph.Scene("served", vols[q["vol"]], tf, vmin, vmax, np.asarray(q["light"]),
                      (1.0, 1.0, 1.0), q["n"], q["R"], q["mode"], q["cam"], q["W"], q["H"],
                      0.5, q["ert"])
        check_frame(out.cpu().numpy(), cnt.cpu().numpy(), oracle_frame(oracle, sc),
                    IMAGE_TOL + FORMAT_HALF_ULP[q["fmt"]])


def test_residency_limit_evicts_and_reloads(env):
    torch, ph, vi, vols, tfs = env
    reqs = make_requests(ph, vi, 12, seed=3)
    alone, _ = run(env, reqs, slots=1, together=False)
    mixed, stats = run(env, reqs, slots=2, together=True, max_resident=1)
    for a, b in zip(alone, mixed):
        assert np.array_equal(a, b)
    assert stats["volume_evictions"] > 0 and stats["volume_loads"] > 3
    assert stats["resident_volumes"] <= 1


def test_request_beyond_the_budget_fails_and_others_finish(env):
    torch, ph, vi, vols, tfs = env
    budget = 64 << 20
    with vi.Server(0, slots=2, memory_budget=budget) as s:
        vid = s.add_volume(vols[0])
        tf, vmin, vmax = tfs[0]
        cam = ph.orbit_camera(np.array([0.3, 0.4, -0.8]), True, 2.4)
        big = torch.empty((16, 16, 4), device="cuda")
        small = torch.empty((16, 16, 4), device="cuda")
        t_big = s.submit(vid, tf, vmin, vmax, (0, 0, 1), 512, 1024, vi.CONE, cam, 16, 16, 0.5, big)
        t_small = s.submit(vid, tf, vmin, vmax, (0, 0, 1), 16, 32, vi.CONE, cam, 16, 16, 0.5, small)
        assert s.wait(t_big) == (vi.REQ_FAILED, vi.ENOMEM)
        assert s.wait(t_small) == (vi.REQ_DONE, vi.OK)
        assert s.stats()["peak_bytes"] <= budget


def test_malformed_requests_are_refused(env):
    torch, ph, vi, vols, tfs = env
    with vi.Server(0, slots=1) as s:
        vid = s.add_volume(vols[0])
        tf, vmin, vmax = tfs[0]
        cam = ph.orbit_camera(np.array([0.3, 0.4, -0.8]), True, 2.4)
        out = torch.empty((8, 8, 4), device="cuda")
        bad_tf = tf.copy()
        bad_tf[3, 3] = 2.0
        for kw in (dict(volume_id=99), dict(tf=bad_tf), dict(light_dir=(0, 0, 0)),
                   dict(n_slices=0), dict(mode=9), dict(vmax=-1.0)):
            args = dict(volume_id=vid, tf=tf, vmin=vmin, vmax=vmax, light_dir=(0, 0, 1),
                        n_slices=8, slice_res=8, mode=vi.SHADOW, cam=cam, W=8, H=8,
                        step_vox=0.5, out=out)
            args.update(kw)
            with pytest.raises(vi.ViError) as e:
                s.submit(**args)
            assert e.value.code == vi.EINVAL
        assert s.stats()["submitted"] == 0


def test_bounded_wait_cancel_and_shutdown(env):
    torch, ph, vi, vols, tfs = env
    s = vi.Server(0, slots=1)
    vid = s.add_volume(vols[1])
    tf, vmin, vmax = tfs[1]
    cam = ph.orbit_camera(np.array([0.3, 0.4, -0.8]), True, 2.4)
    outs = [torch.empty((1024, 1024, 4), device="cuda") for _ in range(3)]
    ts = [s.submit(vid, tf, vmin, vmax, (0.2, 0.1, 1.0), 256, 512, vi.CONE, cam, 1024, 1024,
                   0.25, o) for o in outs]
    with pytest.raises(vi.ViError) as e:     # the last one is still queued behind the others
        s.wait(ts[2], timeout_ms=0.0)
    assert e.value.code == vi.ETIMEOUT
    rc = s.cancel(ts[2])
    assert rc in (vi.OK, vi.ESTATE)
    status, result = s.wait(ts[2])
    assert status == (vi.REQ_CANCELLED if rc == vi.OK else vi.REQ_DONE)
    assert s.wait(ts[0]) == (vi.REQ_DONE, vi.OK)
    t_last = s.submit(vid, tf, vmin, vmax, (0.2, 0.1, 1.0), 256, 512, vi.CONE, cam, 1024, 1024,
                      0.25, outs[2])
    s.close()                                 # cancels what is queued, finishes what runs
    assert s.h is None
    del t_last


def test_kept_stack_serves_a_new_view_of_the_same_scene(env):
    """A second request with the same volume, TF, light and stack but a new
    camera renders from the slot's kept stack: no sweep, same frame as a fresh
    context builds and renders."""
    torch, ph, vi, vols, tfs = env
    tf, vmin, vmax = tfs[1]
    light = (0.3, -0.2, 0.9)
    cams = [ph.orbit_camera(np.array(d), True, 2.4) for d in ((0.3, 0.4, -0.8), (-0.6, 0.1, 0.5))]
    outs = []
    with vi.Server(0, slots=2) as s:
        vid = s.add_volume(vols[1])
        for cam in cams:
            out = torch.empty((40, 48, 4), device="cuda")
            t = s.submit(vid, tf, vmin, vmax, light, 24, 40, vi.CONE, cam, 48, 40, 0.5, out,
                         format=vi.F16, ert=0.95)
            assert s.wait(t) == (vi.REQ_DONE, vi.OK)
            outs.append(out.cpu().numpy())
        assert s.stats()["stack_reuses"] == 1
        # A different TF must not reuse the stack.
        tf2 = tf.copy()
        tf2[:, 3] *= 0.5
        out = torch.empty((40, 48, 4), device="cuda")
        t = s.submit(vid, tf2, vmin, vmax, light, 24, 40, vi.CONE, cams[0], 48, 40, 0.5, out,
                     format=vi.F16, ert=0.95)
        assert s.wait(t) == (vi.REQ_DONE, vi.OK)
        assert s.stats()["stack_reuses"] == 1
    with vi.Context(0) as c:
        c.load_volume(vols[1])
        for cam, got, t_f in ((cams[0], outs[0], tf), (cams[1], outs[1], tf), (cams[0], out.cpu().numpy(), tf2)):
            c.set_transfer_function(t_f, vmin, vmax)
            c.set_light(light)
            c.build_attenuation(24, 40, vi.CONE, format=vi.F16)
            ref = c.render(cam, 48, 40, 0.5, ert=0.95).cpu().numpy()
            assert np.array_equal(got, ref)


def test_threads_submitting_waiting_and_cancelling_concurrently(env):
    """Four host threads submit, wait and sometimes cancel at once: every
    request ends (done or cancelled), no call deadlocks, and every finished
    frame equals the one-at-a-time frame."""
    import threading
    torch, ph, vi, vols, tfs = env
    reqs = make_requests(ph, vi, 24, seed=11)
    alone, _ = run(env, reqs, slots=1, together=False)
    outs = [None] * len(reqs)
    status = [None] * len(reqs)
    errors = []
    with vi.Server(0, slots=3, memory_budget=1 << 30, max_resident_volumes=2) as s:
        vids = [s.add_volume(v) for v in vols]

        def worker(w):
            try:
                rng = np.random.default_rng(100 + w)
                for q_i in range(w, len(reqs), 4):
                    q = reqs[q_i]
                    out = torch.full((q["H"], q["W"], 4), float("nan"), device="cuda")
                    tf, vmin, vmax = tfs[q["vol"]]
                    t = s.submit(vids[q["vol"]], tf, vmin, vmax, q["light"], q["n"], q["R"],
                                 q["mode"], q["cam"], q["W"], q["H"], 0.5, out, format=q["fmt"],
                                 ert=q["ert"])
                    if rng.random() < 0.25:
                        s.cancel(t)           # may already be running: then it completes
                    status[q_i] = s.wait(t, timeout_ms=120000.0)
                    outs[q_i] = out
            except Exception as e:            # surfaced below
                errors.append(repr(e))

        threads = [threading.Thread(target=worker, args=(w,)) for w in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join(timeout=300)
        assert not any(th.is_alive() for th in threads)
        st = s.stats()
    assert not errors, errors
    torch.cuda.synchronize()
    done = 0
    for q_i, (stt, res) in enumerate(status):
        assert (stt, res) in ((vi.REQ_DONE, vi.OK), (vi.REQ_CANCELLED, vi.OK))
        if stt == vi.REQ_DONE:
            assert np.array_equal(outs[q_i].cpu().numpy(), alone[q_i])
            done += 1
    assert done >= 12
    assert st["completed"] == done and st["cancelled"] == len(reqs) - done
    assert st["peak_bytes"] <= 1 << 30


def test_graph_launches_give_the_same_frames(env):
    """With graphs on, each request's sweep, march and output copy run as one
    captured CUDA graph, updated in place for the next request of the same
    shape of work: every frame equals the frame separate launches give, for
    device, page-locked host and pageable host outputs (the last not
    captured), new scenes, a kept-stack view and an unlit frame; one at a
    time and all at once; and a graph is instantiated only when a shape of
    work first appears on a slot."""
    torch, ph, vi, vols, tfs = env
    reqs = make_requests(ph, vi, 20, seed=7)
    again = dict(reqs[3], cam=ph.orbit_camera(np.array((0.2, -0.7, 0.4)), True, 2.4))
    unlit = dict(reqs[5], mode=vi.NONE)
    reqs = reqs[:4] + [again] + reqs[4:] + [unlit]
    kinds = ("device", "pinned", "pageable")
    slots = 3

    def serve(graphs, together):
        with vi.Server(0, slots=slots, graphs=graphs) as s:
            vids = [s.add_volume(v) for v in vols]
            outs, tickets = [], []
            for k, q in enumerate(reqs):
                shape = (q["H"], q["W"], 4)
                kind = kinds[k % 3]
                if kind == "device":
                    out = torch.full(shape, float("nan"), device="cuda")
                elif kind == "pinned":
                    out = torch.full(shape, float("nan")).pin_memory()
                else:
                    out = np.full(shape, np.nan, dtype=np.float32)
                tf, vmin, vmax = tfs[q["vol"]]
                t = s.submit(vids[q["vol"]], tf, vmin, vmax, q["light"], q["n"], q["R"],
                             q["mode"], q["cam"], q["W"], q["H"], 0.5, out, format=q["fmt"],
                             ert=q["ert"])
                outs.append(out)
                tickets.append(t)
                if not together:
                    assert s.wait(t) == (vi.REQ_DONE, vi.OK)
            for t in tickets:
                assert s.wait(t) == (vi.REQ_DONE, vi.OK)
            stats = s.stats()
        torch.cuda.synchronize()
        return [o.cpu().numpy() if hasattr(o, "cpu") else o for o in outs], stats

    captured = sum(kinds[k % 3] != "pageable" for k in range(len(reqs)))
    for together in (False, True):
        ref, st0 = serve(False, together)
        got, st1 = serve(True, together)
        for a, b in zip(ref, got):
            assert np.isfinite(a).all()
            assert np.array_equal(a, b)
        assert st0["graph_launches"] == 0 and st0["graph_instantiations"] == 0
        assert st1["graph_launches"] == captured
        assert 1 <= st1["graph_instantiations"] <= 4 * slots
        if not together:
            assert st0["stack_reuses"] >= 1 and st1["stack_reuses"] == st0["stack_reuses"]


def test_kept_stacks_are_evicted_least_recently_used(env):
    """Two slots, one request at a time: scenes A, B, A (new view), C, A (new
    view).  C replaces the stack used longest ago (B's), so the last view of A
    still renders from A's kept stack: two reuses, and every frame equals the
    frame of a fresh context."""
    torch, ph, vi, vols, tfs = env
    tf, vmin, vmax = tfs[1]
    views = [ph.orbit_camera(np.array(d), True, 2.4)
             for d in ((0.3, 0.4, -0.8), (-0.6, 0.1, 0.5), (0.1, -0.9, 0.2))]
    lights = {"A": (0.3, -0.2, 0.9), "B": (-0.5, 0.4, 0.3), "C": (0.2, 0.8, -0.4)}
    seq = [("A", views[0]), ("B", views[0]), ("A", views[1]), ("C", views[0]), ("A", views[2])]
    got = []
    with vi.Server(0, slots=2) as s:
        vid = s.add_volume(vols[1])
        for scene, cam in seq:
            out = torch.empty((40, 48, 4), device="cuda")
            t = s.submit(vid, tf, vmin, vmax, lights[scene], 24, 40, vi.SHELL, cam, 48, 40,
                         0.5, out)
            assert s.wait(t) == (vi.REQ_DONE, vi.OK)
            got.append(out.cpu().numpy())
        assert s.stats()["stack_reuses"] == 2
    with vi.Context(0) as c:
        c.load_volume(vols[1])
        c.set_transfer_function(tf, vmin, vmax)
        for (scene, cam), frame in zip(seq, got):
            c.set_light(lights[scene])
            c.build_attenuation(24, 40, vi.SHELL)
            assert np.array_equal(frame, c.render(cam, 48, 40, 0.5).cpu().numpy())


def residency_model(seq, costs, max_resident, policy):
    """Loads and evictions of a server admitting the volumes of `seq` one at a
    time with at most `max_resident` resident: LRU, or GreedyDual with the
    reload cost as the cost (credit = clock + cost at each use; the lowest
    credit is evicted, ties by least recent use; the clock rises to the
    victim's credit)."""
    resident, credit, last = set(), {}, {}
    clock, loads, evictions = 0.0, 0, 0
    for t, v in enumerate(seq, start=1):
        if v not in resident:
            while len(resident) >= max_resident:
                if policy == "lru":
                    victim = min(resident, key=lambda u: last[u])
                else:
                    victim = min(resident, key=lambda u: (credit[u], last[u]))
                    clock = max(clock, credit[victim])
                resident.remove(victim)
                evictions += 1
            resident.add(v)
            loads += 1
        last[v] = t
        credit[v] = clock + costs[v]
    return loads, evictions


def test_eviction_policies_follow_their_definitions(env):
    """One request at a time over three volumes with at most two resident: the
    server's loads and evictions equal those of a plain model of each policy
    (GreedyDual on the reload cost, and least recently used), the costly
    volume is reloaded less often under GreedyDual, and the frames do not
    depend on the policy."""
    torch, ph, vi, vols, tfs = env
    rng = np.random.default_rng(21)
    seq = [1, 0, 2, 1] + [int(v) for v in rng.integers(3, size=36)]
    costs = [v.nbytes / float(1 << 20) for v in vols]
    assert max(costs) == costs[1]   # the 48^3 uint16 volume costs most to reload
    cam = ph.orbit_camera(np.array([0.3, -0.5, 0.8]), True, 2.4)
    frames, counts = {}, {}
    for name, policy in (("cost", vi.EVICT_COST), ("lru", vi.EVICT_LRU)):
        with vi.Server(0, slots=2, max_resident_volumes=2, eviction=policy) as s:
            vids = [s.add_volume(v) for v in vols]
            got = []
            for v in seq:
                tf, vmin, vmax = tfs[v]
                out = torch.empty((24, 32, 4), device="cuda")
                t = s.submit(vids[v], tf, vmin, vmax, (0.2, 0.4, -0.9), 8, 16, vi.SHADOW, cam,
                             32, 24, 0.5, out)
                assert s.wait(t) == (vi.REQ_DONE, vi.OK)
                got.append(out.cpu().numpy())
            st = s.stats()
        frames[name] = got
        counts[name] = (st["volume_loads"], st["volume_evictions"])
        assert counts[name] == residency_model(seq, costs, 2, name), name
    for a, b in zip(frames["cost"], frames["lru"]):
        assert np.array_equal(a, b)
    # The first four requests: LRU reloads the costly volume, GreedyDual keeps it.
    assert residency_model(seq[:4], costs, 2, "cost")[0] == 3
    assert residency_model(seq[:4], costs, 2, "lru")[0] == 4
