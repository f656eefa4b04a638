"""GB300-native delta-to-main merge for dictionary-encoded column stores."""
