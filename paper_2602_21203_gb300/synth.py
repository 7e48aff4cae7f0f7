"""Seeded synthetic workloads: configurations and replay-ring contents.

This module holds no arithmetic of the method.  It only names workload shapes
and draws the replay ring (the stand-in for simulator frames), so that the
CUDA path and the FP64 oracle can be fed identical inputs.

Distributions (stand-ins for wrist-camera frames and proprioception of the
SO-101 tasks, Sec. V): obs uint8 uniform on [0, 255], proprio ~ N(0, 1),
action ~ U(-1, 1), reward ~ N(0, 1), done ~ Bernoulli(0.02).
"""
import copy

import torch

_COMMON = dict(
    obs_c=3, proprio_dim=12, action_dim=6, n_critics=2,
    gamma=0.99, lr=3e-4, tau=0.005, init_alpha=0.1, target_entropy=None,
    policy_freq=1, seed=0, ln_eps=1e-5, log_std_min=-5.0, log_std_max=2.0,
    adam_b1=0.9, adam_b2=0.999, adam_eps=1e-8, conv_strides=None,
)

PRESETS = {
    # Single FP32 update on a small ring: 256 slots of 3x64x64, batch 32,
    # shift pad 4, squint 4x to 16x16, 2 conv layers of 16 channels (stride 2, 1),
    # no projection, critics/actor 256-256, 51 atoms on [-10, 10].
    "small_b32": dict(ring_size=256, obs_h=64, obs_w=64, squint_f=4, shift_pad=4, batch=32,
                      conv_layers=2, conv_ch=16, proj_dim=0, hidden=[256, 256],
                      atoms=51, v_min=-10.0, v_max=10.0, utd=1),
    # Training shape: 100k slots of 3x128x128 (4.9 GB), batch 512, shift pad 8,
    # squint 4x to 32x32, 4 conv layers of 32 channels, 256-d projection + LN,
    # critics 512-512 x2 with 101 atoms on [-20, 20], actor 512-512, 4 updates per call.
    "train_b512": dict(ring_size=100_000, obs_h=128, obs_w=128, squint_f=4, shift_pad=8, batch=512,
                       conv_layers=4, conv_ch=32, proj_dim=256, hidden=[512, 512],
                       atoms=101, v_min=-20.0, v_max=20.0, utd=4),
    # Squint at insert (the paper's replay layout, Alg. 1): 1M slots of squinted
    # 3x32x32 uint8 frames (3 GB), filled by squint_op_squint_store from 3x128x128
    # renders, read with f = 1 and the shift at 32x32 (pad 2 = 8 / 4); same networks as
    # train_b512.
    "stored_b512": dict(ring_size=1_000_000, obs_h=32, obs_w=32, squint_f=1, shift_pad=2, batch=512,
                        conv_layers=4, conv_ch=32, proj_dim=256, hidden=[512, 512],
                        atoms=101, v_min=-20.0, v_max=20.0, utd=4, render_h=128, render_w=128, render_f=4),
    # State-based SAC (Sec. VII, Fig. 6 left: the encoder removed): 1M slots of a 48-d
    # state vector, batch 512, the same critics / actor (512-512, 101 atoms on [-20, 20])
    # and UTD 4 as train_b512; no image in the ring.
    "state_b512": dict(ring_size=1_000_000, obs_c=0, obs_h=0, obs_w=0, squint_f=1, shift_pad=0, batch=512,
                       proprio_dim=48, conv_layers=0, conv_ch=0, proj_dim=0, hidden=[512, 512],
                       atoms=101, v_min=-20.0, v_max=20.0, utd=4),
    # Small state-based case for parity: 512 slots of a 20-d state, batch 64, MLPs 256-256.
    "state_small_b64": dict(ring_size=512, obs_c=0, obs_h=0, obs_w=0, squint_f=1, shift_pad=0, batch=64,
                            proprio_dim=20, conv_layers=0, conv_ch=0, proj_dim=0, hidden=[256, 256],
                            atoms=51, v_min=-10.0, v_max=10.0, utd=4),
    # Tiny net for finite differences: 3x64x64 ring squinted to 3x16x16, 8 channels,
    # MLPs 32-32, 11 atoms on [-10, 10] (atom spacing exactly 2), batch 8.
    "tiny_b8": dict(ring_size=64, obs_h=64, obs_w=64, squint_f=4, shift_pad=4, batch=8,
                    conv_layers=2, conv_ch=8, proj_dim=0, hidden=[32, 32],
                    atoms=11, v_min=-10.0, v_max=10.0, utd=8),
}


def make_config(name, **overrides):
    """A workload configuration (plain dict) from a preset name plus overrides."""
    cfg = copy.deepcopy(_COMMON)
    cfg.update(copy.deepcopy(PRESETS[name]))
    cfg.update(overrides)
    return cfg


def make_ring(cfg, seed=0, device="cpu"):
    """Replay ring contents as torch tensors on `device` (seeded; device decides the stream)."""
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    n, c, h, w = cfg["ring_size"], cfg["obs_c"], cfg["obs_h"], cfg["obs_w"]
    state_based = cfg["conv_layers"] == 0          # no image in the ring
    obs = None if state_based else torch.randint(0, 256, (n, c, h, w), dtype=torch.uint8, generator=g, device=device)
    proprio = torch.randn(n, cfg["proprio_dim"], generator=g, device=device)
    action = torch.rand(n, cfg["action_dim"], generator=g, device=device) * 2.0 - 1.0
    reward = torch.randn(n, generator=g, device=device)
    done = (torch.rand(n, generator=g, device=device) < 0.02).to(torch.uint8)
    ring = dict(proprio=proprio, action=action, reward=reward, done=done)
    if not state_based:
        ring["obs"] = obs
    return ring


def render_frames(n, cfg, seed, device="cpu"):
    """Seeded uint8 renders [n, C, render_h, render_w] for a squint-at-insert workload."""
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.randint(0, 256, (n, cfg["obs_c"], cfg["render_h"], cfg["render_w"]), dtype=torch.uint8,
                         generator=g, device=device)


def ring_numpy(ring):
    """Host numpy copies of a ring (what the oracle reads)."""
    return {k: v.detach().cpu().numpy() for k, v in ring.items()}


def make_obs_batch(n, cfg, seed, device="cpu"):
    """Inference inputs for n environments: uint8 frames at render resolution and proprio."""
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    obs = None
    if cfg["conv_layers"] > 0:
        obs = torch.randint(0, 256, (n, cfg["obs_c"], cfg["obs_h"], cfg["obs_w"]), dtype=torch.uint8,
                            generator=g, device=device)
    prop = torch.randn(n, cfg["proprio_dim"], generator=g, device=device)
    return obs, prop
